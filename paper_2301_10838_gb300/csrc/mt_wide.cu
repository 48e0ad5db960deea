// Triplet merge trees with wide vertex ids (grids of 2^32 vertices and more).
//
// Section 3.2 of the paper packs the two 32-bit ids of a triplet (s, v) into
// one 64-bit word because SYCL offers no double-word compare-and-swap, which
// caps a grid at 2^32 vertices; Section 5 names wider ids as future work. On
// sm_103a a 128-bit compare-and-swap exists (atom.cas.b128), so this path
// keeps the whole triplet in one 128-bit word, W[u] = (s, v) with two 64-bit
// ids. It computes the same unique triplets as the 32-bit path, in three
// steps of Algorithm 1 (which merges the edges in any order):
//   1. the tile kernel of the 32-bit path (mt_build.cu) builds the merge tree
//      of every 32x16x16 tile in shared memory on 16-bit local ids and writes
//      it with 64-bit ids (launch_tile_wide);
//   2. k_w_cross merges every edge between neighbouring tiles with the
//      lock-free Merge (Algorithms 2 and 3) on the global 128-bit words,
//      starting from the edge's two ends;
//   3. k_w_repair restores minimality (Algorithms 4 and 5).
//
// Torn reads. While merges run, every 64-bit half of a word carries the same
// 30-bit version tag above its 34-bit id; a compare-and-swap writes both
// halves with the next tag. A reader that loads the two halves and finds
// different tags saw a concurrent update between them and loads again, so a
// climb never follows a pair (s, v) that no Merge wrote, whatever the
// hardware's atomicity for 128-bit loads. Ids therefore have 34 bits:
// n < 2^34 vertices, more than fit in the 288 GB of one GB300 at the 20 bytes
// per vertex the field and the triplets take. The tile kernel writes tag 0;
// repair writes every word back without its tag.
//
// Pairs and labels: k_w_pairs_count / k_w_scan / k_w_pairs_write (ordered
// compaction with 64-bit offsets) and k_w_labels (a chase per vertex).
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/mt.h"
#include "mt_device.cuh"
#include "mt_internal.h"

namespace mt {
namespace {

constexpr uint32_t kIdBits = 34;
constexpr uint64_t kIdMask = (1ull << kIdBits) - 1;
constexpr uint64_t kMaxWideVertices = 1ull << kIdBits;
constexpr uint32_t kTagMask = (1u << (64 - kIdBits)) - 1;
constexpr uint32_t kWChunk = 4096;         // vertices per pair-compaction chunk
constexpr int kWThreads = 256;

// Workspace: [0, 256) status word, [256, 512) meta (npairs, roots, root),
// then per-chunk pair counts (u32) and offsets (u64).
struct WideWs {
    uint32_t *status;
    uint64_t *meta;
    uint32_t *counts;
    uint64_t *offsets;
    uint64_t nchunks;
};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t wide_ws_bytes(uint64_t n)
{
    const uint64_t nchunks = (n + kWChunk - 1) / kWChunk;
    return 512 + al256(nchunks * 4) + al256(nchunks * 8);
}

bool carve(void *base, size_t bytes, uint64_t n, WideWs &ws)
{
    if (!base || ((uintptr_t)base & 255) || bytes < wide_ws_bytes(n)) return false;
    char *p = static_cast<char *>(base);
    ws.nchunks = (n + kWChunk - 1) / kWChunk;
    ws.status = reinterpret_cast<uint32_t *>(p);
    ws.meta = reinterpret_cast<uint64_t *>(p + 256);
    ws.counts = reinterpret_cast<uint32_t *>(p + 512);
    ws.offsets = reinterpret_cast<uint64_t *>(p + 512 + al256(ws.nchunks * 4));
    return true;
}

struct Geo {
    uint64_t nx, ny, nz, nxy, n;
};

// the values as the order sees them (sg = -1: the tree of -f)
struct FieldW {
    const float *f;
    float sg;
    __device__ __forceinline__ float operator[](uint64_t i) const { return sg * __ldg(f + i); }
};

__device__ __forceinline__ bool before_w(float fa, uint64_t a, float fb, uint64_t b)
{
    return fa < fb || (fa == fb && a < b);
}

// 128-bit compare-and-swap of the word at p (two u64: lo, hi); returns the old word.
__device__ __forceinline__ void cas128(uint64_t *p, uint64_t cmp_lo, uint64_t cmp_hi, uint64_t new_lo,
                                       uint64_t new_hi, uint64_t &old_lo, uint64_t &old_hi)
{
    asm volatile("{\n\t.reg .b128 c, w, o;\n\t"
                 "mov.b128 c, {%2, %3};\n\t"
                 "mov.b128 w, {%4, %5};\n\t"
                 "atom.relaxed.gpu.global.cas.b128 o, [%6], c, w;\n\t"
                 "mov.b128 {%0, %1}, o;\n\t}"
                 : "=l"(old_lo), "=l"(old_hi)
                 : "l"(cmp_lo), "l"(cmp_hi), "l"(new_lo), "l"(new_hi), "l"(p)
                 : "memory");
}

// Both halves of a word in one 16-byte load (one memory sector); the
// memory model guarantees each 8-byte half, not the pair.
__device__ __forceinline__ void ld_word(const uint64_t *W, uint64_t u, uint64_t &lo, uint64_t &hi)
{
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(lo), "=l"(hi) : "l"(W + 2 * u) : "memory");
}

// A word read during the merges: both halves with the same tag. Returns
// false if every one of a bounded number of reads was torn.
__device__ __forceinline__ bool wload(const uint64_t *W, uint64_t u, uint64_t &lo, uint64_t &hi)
{
    for (int i = 0; i < 1024; i++) {
        ld_word(W, u, lo, hi);
        if ((lo >> kIdBits) == (hi >> kIdBits)) return true;
    }
    return false;
}

// ----------------------------------------------------------------- merge
// Climb (Algorithm 3): from x, follow links whose saddle is at or below
// (fS, S) in the order; a root stops the walk. Returns false if a read
// stayed torn or the step budget ran out.
struct WideMerge {
    uint64_t *W;
    FieldW f;

    __device__ __forceinline__ bool climb(uint64_t &x, uint64_t S, float fS, uint64_t &lo, uint64_t &hi,
                                          uint32_t &steps) const
    {
        if (!wload(W, x, lo, hi)) return false;
        for (;;) {
            const uint64_t s = lo & kIdMask, v = hi & kIdMask;
            if (s == x && v == x) return true;
            if (s != S && !before_w(f[s], s, fS, S)) return true;
            x = v;
            if (!wload(W, x, lo, hi) || ++steps > kMergeStepLimit) return false;
        }
    }

    // Merge(S, a, b): make a and b connected at level S (Algorithm 3).
    __device__ bool merge(uint64_t S, uint64_t a, uint64_t b) const
    {
        float fS = f[S];
        uint64_t u = a, v = b;
        uint32_t steps = 0;
        for (;;) {
            uint64_t ulo, uhi, vlo, vhi;
            if (!climb(u, S, fS, ulo, uhi, steps) || !climb(v, S, fS, vlo, vhi, steps)) return false;
            if (++steps > kMergeStepLimit) return false;
            if (u == v) return true;
            if (before_w(f[v], v, f[u], u)) {
                uint64_t t = u;
                u = v, v = t;
                t = ulo, ulo = vlo, vlo = t;
                t = uhi, uhi = vhi, vhi = t;
            }
            const uint64_t tag = (uint64_t)(((vlo >> kIdBits) + 1) & kTagMask) << kIdBits;
            uint64_t olo, ohi;
            cas128(W + 2 * v, vlo, vhi, S | tag, u | tag, olo, ohi);
            if (olo == vlo && ohi == vhi) {
                const uint64_t sv = vlo & kIdMask, tv = vhi & kIdMask;
                if (sv == v && tv == v) return true;  // displaced a root: it carries no link
                S = sv;                                // re-insert the displaced link
                fS = f[sv];
                v = tv;
            }
        }
    }
};

// One CTA per 32x16x16 tile: the edges from the tile to its +x, +y and +z
// neighbour tiles, each merged from its two ends at the level of its later
// end (the tile kernel has already merged every edge inside a tile).
constexpr uint32_t kTX = 32, kTY = 16, kTZ = 16;

__global__ void __launch_bounds__(256) k_w_cross(FieldW f, Geo g, uint32_t ntx, uint32_t nty, uint64_t *W,
                                                 uint32_t *status)
{
    if (*status) return;  // no barriers below: a per-thread test is enough
    constexpr uint32_t FX = kTY * kTZ, FY = kTX * kTZ, FZ = kTX * kTY, FH = FX + FY + FZ;
    const WideMerge M{W, f};
    const uint32_t tile = blockIdx.x;
    const uint32_t tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
    const uint64_t x0 = (uint64_t)tx * kTX, y0 = (uint64_t)ty * kTY, z0 = (uint64_t)tz * kTZ;
    const uint64_t wx = min((uint64_t)kTX, g.nx - x0), wy = min((uint64_t)kTY, g.ny - y0),
                   wz = min((uint64_t)kTZ, g.nz - z0);
    const uint64_t base = z0 * g.nxy + y0 * g.nx + x0;
    const bool hx = x0 + kTX < g.nx, hy = y0 + kTY < g.ny, hz = z0 + kTZ < g.nz;
    bool ok = true;
    for (uint32_t e = threadIdx.x; e < FH; e += blockDim.x) {
        uint64_t a, b;
        if (e < FX) {
            const uint64_t ly = e % kTY, lz = e / kTY;
            if (!hx || ly >= wy || lz >= wz) continue;
            a = base + lz * g.nxy + ly * g.nx + (kTX - 1);
            b = a + 1;
        } else if (e < FX + FY) {
            const uint64_t k = e - FX, lx = k % kTX, lz = k / kTX;
            if (!hy || lx >= wx || lz >= wz) continue;
            a = base + lz * g.nxy + (kTY - 1) * g.nx + lx;
            b = a + g.nx;
        } else {
            const uint64_t k = e - FX - FY, lx = k % kTX, ly = k / kTX;
            if (!hz || lx >= wx || ly >= wy) continue;
            a = base + (kTZ - 1) * g.nxy + ly * g.nx + lx;
            b = a + g.nxy;
        }
        const uint64_t S = before_w(f[a], a, f[b], b) ? b : a;
        ok &= M.merge(S, a, b);
    }
    if (!ok) raise_status(status, ST_TIMEOUT);
}

// ---------------------------------------------------------------- repair
// Representative (Algorithm 4) at level S: hop while the link's saddle is at
// or below S in the order; return the vertex where the walk stops. Concurrent
// repairs only move a word's target further along its own chain below the
// same saddle, so either half may be old or new. The next word is read
// beside the saddle's value, before the test that decides whether it is
// needed (the target of a link is a vertex of the grid, so the read stays in
// bounds); the same in the climbs of the merges, whose reads repeat until
// both halves carry one tag, measured slower.
__device__ __forceinline__ uint64_t w_rep(const uint64_t *W, const FieldW &f, uint64_t x, uint64_t S, float fS,
                                          uint32_t &steps)
{
    uint64_t lo, hi;
    ld_word(W, x, lo, hi);
    for (;;) {
        const uint64_t s = lo & kIdMask, v = hi & kIdMask;
        if (s == x && v == x) return x;
        const float fs = f[s];
        uint64_t nlo, nhi;
        ld_word(W, v, nlo, nhi);
        if (s != S && !before_w(fs, s, fS, S)) return x;
        x = v, lo = nlo, hi = nhi;
        if (++steps > kChaseLimit) return x;
    }
}

__global__ void __launch_bounds__(kWThreads) k_w_repair(FieldW f, Geo g, uint64_t *W, uint32_t *status)
{
    if (*status) return;
    bool ok = true;
    for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < g.n; u += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t lo, hi;
        ld_word(W, u, lo, hi);
        const uint64_t s = lo & kIdMask, v = hi & kIdMask;
        uint64_t r = v;
        if (!(s == u && v == u)) {
            uint32_t steps = 0;
            // a minimum: its target at its saddle s; an inner vertex: at u itself
            r = w_rep(W, f, v, s, f[s], steps);
            if (steps > kChaseLimit) {
                ok = false;
                continue;
            }
        }
        if (r != v || lo != s || hi != v)
            asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(W + 2 * u), "l"(s), "l"(r) : "memory");
    }
    if (!ok) raise_status(status, ST_TIMEOUT);
}

// ----------------------------------------------------------------- pairs
__global__ void __launch_bounds__(kWThreads) k_w_pairs_count(const uint64_t *W, uint64_t n, uint32_t *counts,
                                                             uint64_t *meta, const uint32_t *status)
{
    if (block_skips(status)) return;
    __shared__ uint32_t s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const uint64_t a = blockIdx.x * (uint64_t)kWChunk;
    uint32_t c = 0;
    for (uint64_t u = a + threadIdx.x; u < a + kWChunk && u < n; u += kWThreads) {
        const uint64_t s = W[2 * u], v = W[2 * u + 1];
        if (s != u) {
            c++;
        } else if (v == u) {
            atomicAdd(reinterpret_cast<unsigned long long *>(meta + 1), 1ull);
            meta[2] = u;
        }
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&s_cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) counts[blockIdx.x] = s_cnt;
}

// exclusive scan of the chunk counts into 64-bit offsets (one CTA): warp w
// owns a contiguous range read in coalesced rows of 32; a pass sums the
// ranges, one warp scans the sums, and a second pass scans row by row with
// shuffles on top of the carry
__global__ void __launch_bounds__(1024) k_w_scan(const uint32_t *counts, uint64_t *offsets, uint64_t m,
                                                 uint64_t *meta, const uint32_t *status)
{
    if (block_skips(status)) return;
    __shared__ uint64_t wsum[32];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t per = ((m + 31) / 32 + 31) / 32 * 32;
    const uint64_t a = warp * per, b = a + per < m ? a + per : m;
    uint64_t s = 0;
    for (uint64_t i = a + lane; i < b; i += 32) s += counts[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) wsum[warp] = s;
    __syncthreads();
    if (warp == 0) {
        const uint64_t v = wsum[lane];
        uint64_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        wsum[lane] = incl - v;
        if (lane == 31) meta[0] = incl;
    }
    __syncthreads();
    uint64_t carry = wsum[warp];
    for (uint64_t r = a; r < b; r += 32) {
        const uint64_t i = r + lane;
        const uint32_t c = i < b ? counts[i] : 0u;
        uint32_t incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        if (i < b) offsets[i] = carry + incl - c;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
}

// ordered write: the chunk's pairs at its offset, by ascending u (one warp
// after another, ballots rank the lanes)
__global__ void __launch_bounds__(kWThreads) k_w_pairs_write(const uint64_t *W, uint64_t n, const uint64_t *offsets,
                                                             uint64_t *pairs, uint64_t cap, const uint32_t *status)
{
    if (block_skips(status)) return;
    constexpr int kWarps = kWThreads / 32;
    constexpr uint32_t kPerWarp = kWChunk / kWarps;
    __shared__ uint32_t s_wc[kWarps];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t a = blockIdx.x * (uint64_t)kWChunk + (uint64_t)warp * kPerWarp;
    uint32_t c = 0;
    for (uint32_t r = 0; r < kPerWarp; r += 32) {
        const uint64_t u = a + r + lane;
        const bool p = u < n && W[2 * u] != u;
        c += __popc(__ballot_sync(0xffffffffu, p));
    }
    if (lane == 0) s_wc[warp] = c;
    __syncthreads();
    uint64_t run = offsets[blockIdx.x];
    for (uint32_t w = 0; w < warp; w++) run += s_wc[w];
    for (uint32_t r = 0; r < kPerWarp; r += 32) {
        const uint64_t u = a + r + lane;
        const uint64_t s = u < n ? W[2 * u] : u;
        const bool p = u < n && s != u;
        const uint32_t ball = __ballot_sync(0xffffffffu, p);
        if (p) {
            const uint64_t pos = run + __popc(ball & ((1u << lane) - 1u));
            if (pos < cap) pairs[2 * pos] = u, pairs[2 * pos + 1] = s;
        }
        run += __popc(ball);
    }
}

// ---------------------------------------------------------------- labels
// label[u] = the deepest vertex of u's component of G_t (Algorithm 4 with the
// value test f(s) <= t), or all ones when f[u] > t.
__global__ void __launch_bounds__(kWThreads) k_w_labels(FieldW f, uint64_t n, const uint64_t *W, float t,
                                                        uint64_t *labels, uint32_t *status)
{
    if (*status) return;
    bool ok = true, bad = false;
    for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < n; u += (uint64_t)gridDim.x * blockDim.x) {
        if (!(f[u] <= t)) {
            labels[u] = ~0ull;
            continue;
        }
        const ulonglong2 wu = reinterpret_cast<const ulonglong2 *>(W)[u];
        uint64_t x = (wu.x == u && wu.y != u) ? wu.y : u;
        for (uint64_t h = 0;; h++) {
            const ulonglong2 wx = reinterpret_cast<const ulonglong2 *>(W)[x];
            const uint64_t s = wx.x, v = wx.y;
            if (s == x && v == x) break;
            if (s >= n || v >= n) {
                bad = true;
                break;
            }
            if (!(f[s] <= t)) break;
            x = v;
            if (h >= kChaseLimit || h >= n) {
                ok = false;
                break;
            }
        }
        labels[u] = x;
    }
    if (!ok) raise_status(status, ST_TIMEOUT);
    if (bad) raise_status(status, ST_CORRUPT);
}

unsigned grid_for(uint64_t work)
{
    const uint64_t per_block = kWThreads * 8ull;
    const uint64_t want = (work + per_block - 1) / per_block;
    const uint64_t cap = (uint64_t)device_sms() * 16;
    return (unsigned)(want < 1 ? 1 : want > cap ? cap : want);
}

mt_status wide_grid(mt_grid g, Geo &geo)
{
    if (g.nx == 0 || g.ny == 0 || g.nz == 0) return MT_ERR_INVALID;
    geo.nx = g.nx, geo.ny = g.ny, geo.nz = g.nz;
    geo.nxy = geo.nx * geo.ny;
    geo.n = geo.nxy * geo.nz;
    if (geo.n >= kMaxWideVertices) return MT_ERR_TOO_LARGE;
    return MT_OK;
}

}  // namespace
}  // namespace mt

using namespace mt;

extern "C" {

size_t mt_wide_workspace_bytes(mt_grid g)
{
    Geo geo;
    if (wide_grid(g, geo) != MT_OK) return 0;
    return wide_ws_bytes(geo.n);
}

mt_status mt_build_triplets_wide(const float *d_f, mt_grid g, uint64_t *d_W, void *d_ws, size_t ws_bytes,
                                 uint32_t flags, void *stream)
{
    Geo geo;
    mt_status st = wide_grid(g, geo);
    if (st != MT_OK) return st;
    if (!d_f || !d_W || ((uintptr_t)d_f & 3) || ((uintptr_t)d_W & 15) || (flags & ~MT_SUPERLEVEL))
        return MT_ERR_INVALID;
    WideWs ws;
    if (!carve(d_ws, ws_bytes, geo.n, ws)) return MT_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float sg = (flags & MT_SUPERLEVEL) ? -1.0f : 1.0f;
    const FieldW f{d_f, sg};
    if (cudaMemsetAsync(ws.status, 0, 512, s) != cudaSuccess) return MT_ERR_CUDA;
    {
        PhaseScope ps(kTile, s);
        if (launch_tile_wide(d_f, d_W, g.nx, g.ny, g.nz, sg, ws.status, s) != cudaSuccess) return MT_ERR_CUDA;
    }
    const uint32_t ntx = (g.nx + kTX - 1) / kTX, nty = (g.ny + kTY - 1) / kTY, ntz = (g.nz + kTZ - 1) / kTZ;
    {
        PhaseScope ps(kMerge, s);
        k_w_cross<<<ntx * nty * ntz, 256, 0, s>>>(f, geo, ntx, nty, d_W, ws.status);
        count_launch();
    }
    {
        PhaseScope ps(kRepair, s);
        k_w_repair<<<grid_for(geo.n), kWThreads, 0, s>>>(f, geo, d_W, ws.status);
        count_launch();
    }
    return cudaGetLastError() == cudaSuccess ? MT_OK : MT_ERR_CUDA;
}

mt_status mt_persistence_pairs_wide(const uint64_t *d_W, mt_grid g, uint64_t *d_pairs, uint64_t cap,
                                    uint64_t *h_npairs, uint64_t *h_root, void *d_ws, size_t ws_bytes, void *stream)
{
    Geo geo;
    mt_status st = wide_grid(g, geo);
    if (st != MT_OK) return st;
    if (!d_W || !h_npairs || ((uintptr_t)d_W & 15) || (cap && (!d_pairs || ((uintptr_t)d_pairs & 7))))
        return MT_ERR_INVALID;
    WideWs ws;
    if (!carve(d_ws, ws_bytes, geo.n, ws)) return MT_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(ws.meta, 0, 3 * sizeof(uint64_t), s) != cudaSuccess) return MT_ERR_CUDA;
    {
        PhaseScope ps(kPairs, s);
        k_w_pairs_count<<<(unsigned)ws.nchunks, kWThreads, 0, s>>>(d_W, geo.n, ws.counts, ws.meta, ws.status);
        k_w_scan<<<1, 1024, 0, s>>>(ws.counts, ws.offsets, ws.nchunks, ws.meta, ws.status);
        k_w_pairs_write<<<(unsigned)ws.nchunks, kWThreads, 0, s>>>(d_W, geo.n, ws.offsets, d_pairs, cap,
                                                                   ws.status);
        count_launch(3);
        if (cudaGetLastError() != cudaSuccess) return MT_ERR_CUDA;
    }
    uint64_t meta[4];
    if (readback(ws.meta, ws.status, s, meta) != cudaSuccess) return MT_ERR_CUDA;
    const uint32_t bits = (uint32_t)meta[3];
    if (bits) return status_from_bits(bits);
    *h_npairs = meta[0];
    if (h_root) *h_root = meta[1] == 1 ? meta[2] : ~0ull;
    if (meta[1] != 1) return MT_ERR_INVALID;
    return meta[0] > cap ? MT_ERR_CAPACITY : MT_OK;
}

mt_status mt_components_at_wide(const float *d_f, const uint64_t *d_W, mt_grid g, float t, uint32_t flags,
                                uint64_t *d_labels, void *d_ws, size_t ws_bytes, void *stream)
{
    Geo geo;
    mt_status st = wide_grid(g, geo);
    if (st != MT_OK) return st;
    if (!d_f || !d_W || !d_labels || std::isnan(t) || ((uintptr_t)d_f & 3) || ((uintptr_t)d_W & 15) ||
        ((uintptr_t)d_labels & 7) || (flags & ~MT_SUPERLEVEL))
        return MT_ERR_INVALID;
    WideWs ws;
    if (!carve(d_ws, ws_bytes, geo.n, ws)) return MT_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float sg = (flags & MT_SUPERLEVEL) ? -1.0f : 1.0f;
    PhaseScope ps(kLabels, s);
    k_w_labels<<<grid_for(geo.n), kWThreads, 0, s>>>(FieldW{d_f, sg}, geo.n, d_W, sg * t, d_labels, ws.status);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? MT_OK : MT_ERR_CUDA;
}

}  // extern "C"
