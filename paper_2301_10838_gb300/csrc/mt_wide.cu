// Triplet merge trees with wide vertex ids (grids of 2^32 vertices and more).
//
// Section 3.2 of the paper packs the two 32-bit ids of a triplet (s, v) into
// one 64-bit word because SYCL offers no double-word compare-and-swap, which
// caps a grid at 2^32 vertices; Section 5 names wider ids as future work. On
// sm_103a a 128-bit compare-and-swap exists (atom.cas.b128), so this path
// keeps the whole triplet in one 128-bit word, W[u] = (s, v) with two 64-bit
// ids, and otherwise runs Algorithm 1 as written: every vertex is seeded with
// its lowest lower neighbour, every edge is merged with the lock-free Merge
// (Algorithms 2 and 3) on global memory, and Repair (Algorithms 4 and 5)
// restores minimality. It computes the same unique triplets as the 32-bit
// path, only with 64-bit ids; it does not use the tiled shared-memory merges
// of that path.
//
// Torn reads. While merges run, every 64-bit half of a word carries the same
// 30-bit version tag above its 34-bit id; a compare-and-swap writes both
// halves with the next tag. A reader that loads the two halves and finds
// different tags saw a concurrent update between them and loads again, so a
// climb never follows a pair (s, v) that no Merge wrote, whatever the
// hardware's atomicity for 128-bit loads. Ids therefore have 34 bits:
// n < 2^34 vertices, more than fit in the 288 GB of one GB300 at the 20 bytes
// per vertex the field and the triplets take. Repair writes every word back
// without its tag.
//
// Kernels (one thread per vertex or per edge, grid-stride over 64-bit ranges):
//   k_w_init     validate, seed W[u] = (u, lowest lower neighbour) or (u, u)
//   k_w_jump     pointer doubling along the descent links (a fixed number of
//                passes, each a no-op once the previous one changed nothing)
//   k_w_merge    Merge of every edge whose ends descend to different minima
//   k_w_repair   Repair, writing the final untagged words
//   k_w_pairs_count / k_w_scan / k_w_pairs_write   ordered pair compaction
//   k_w_labels   components at a threshold
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
constexpr int kJumpPasses = kIdBits + 2;  // doubling: chains shorter than 2^34 converge in 34 passes
constexpr uint32_t kWChunk = 4096;         // vertices per pair-compaction chunk
constexpr int kWThreads = 256;

// Workspace: [0, 256) status word, [256, 512) meta (npairs, roots, root),
// [512, 768) jump flags (one u32 per pass), then per-chunk pair counts (u32)
// and offsets (u64).
struct WideWs {
    uint32_t *status;
    uint64_t *meta;
    uint32_t *jflag;
    uint32_t *counts;
    uint64_t *offsets;
    uint64_t nchunks;
};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t wide_ws_bytes(uint64_t n)
{
    const uint64_t nchunks = (n + kWChunk - 1) / kWChunk;
    return 768 + al256(nchunks * 4) + al256(nchunks * 8);
}

bool carve(void *base, size_t bytes, uint64_t n, WideWs &ws)
{
    if (!base || ((uintptr_t)base & 255) || bytes < wide_ws_bytes(n)) return false;
    char *p = static_cast<char *>(base);
    ws.nchunks = (n + kWChunk - 1) / kWChunk;
    ws.status = reinterpret_cast<uint32_t *>(p);
    ws.meta = reinterpret_cast<uint64_t *>(p + 256);
    ws.jflag = reinterpret_cast<uint32_t *>(p + 512);
    ws.counts = reinterpret_cast<uint32_t *>(p + 768);
    ws.offsets = reinterpret_cast<uint64_t *>(p + 768 + al256(ws.nchunks * 4));
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

__device__ __forceinline__ uint64_t ld_rel(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
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

// A word read during the merges: both halves with the same tag. Returns
// false if every one of a bounded number of reads was torn.
__device__ __forceinline__ bool wload(const uint64_t *W, uint64_t u, uint64_t &lo, uint64_t &hi)
{
    for (int i = 0; i < 1024; i++) {
        lo = ld_rel(W + 2 * u);
        hi = ld_rel(W + 2 * u + 1);
        if ((lo >> kIdBits) == (hi >> kIdBits)) return true;
    }
    return false;
}

__device__ __forceinline__ void wcoords(const Geo &g, uint64_t u, uint64_t &x, uint64_t &y, uint64_t &z)
{
    x = u % g.nx;
    const uint64_t r = u / g.nx;
    y = r % g.ny;
    z = r / g.ny;
}

// ------------------------------------------------------------------ init
__global__ void __launch_bounds__(kWThreads) k_w_init(FieldW f, Geo g, uint64_t *W, uint32_t *status)
{
    bool bad = false;
    for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < g.n; u += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t x, y, z;
        wcoords(g, u, x, y, z);
        const float fu = f[u];
        bad |= !isfinite(fu);
        uint64_t b = u;
        float fb = fu;
        // lowest lower neighbour in the order (value, index)
        const uint64_t cand[6] = {x > 0 ? u - 1 : u, x + 1 < g.nx ? u + 1 : u, y > 0 ? u - g.nx : u,
                                  y + 1 < g.ny ? u + g.nx : u, z > 0 ? u - g.nxy : u, z + 1 < g.nz ? u + g.nxy : u};
#pragma unroll
        for (int k = 0; k < 6; k++) {
            const uint64_t w = cand[k];
            if (w == u) continue;
            const float fw = f[w];
            if (before_w(fw, w, fb, b)) b = w, fb = fw;
        }
        W[2 * u] = u;      // s = u, tag 0
        W[2 * u + 1] = b;  // v = lowest lower neighbour, or u
    }
    if (bad) raise_status(status, ST_NONFINITE);
}

// ------------------------------------------------------------------ jump
// Pass p: every inner vertex u (W[u] = (u, v), v != u) replaces v by the
// target of v, up to four times; concurrent replacements only move targets
// further down the same descent path, so any value read is valid. A pass
// after one that changed nothing returns at once.
__global__ void __launch_bounds__(kWThreads) k_w_jump(Geo g, uint64_t *W, uint32_t *jflag, int pass,
                                                      const uint32_t *status)
{
    if (__syncthreads_or(threadIdx.x == 0 && (*(const volatile uint32_t *)status != 0 ||
                                              (pass > 0 && jflag[pass - 1] == 0))))
        return;
    bool changed = false;
    for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < g.n; u += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v0 = ld_rel(W + 2 * u + 1);
        if (v0 == u) continue;
        uint64_t v = v0;
        for (int k = 0; k < 4; k++) {
            const uint64_t w = ld_rel(W + 2 * v + 1);
            if (w == v) break;
            v = w;
        }
        if (v != v0) {
            asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(W + 2 * u + 1), "l"(v) : "memory");
            changed = true;
        }
    }
    if (__syncthreads_or(changed) && threadIdx.x == 0) atomicOr(jflag + pass, 1u);
}

__global__ void k_w_jump_check(const uint32_t *jflag, uint32_t *status)
{
    if (jflag[kJumpPasses - 1]) raise_status(status, ST_TIMEOUT);
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

// One thread per (vertex, direction +x/+y/+z). Inner vertices keep their
// word (u, minimum) through the merges, so the minimum an end descends to is
// read once; an edge whose ends descend to the same minimum is skipped.
__global__ void __launch_bounds__(kWThreads) k_w_merge(FieldW f, Geo g, uint64_t *W, uint32_t *status)
{
    if (*status) return;
    const WideMerge M{W, f};
    bool ok = true;
    const uint64_t ne = 3 * g.n;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < ne; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t u = e / 3;
        const uint32_t d = (uint32_t)(e - 3 * u);
        uint64_t x, y, z;
        wcoords(g, u, x, y, z);
        uint64_t w;
        if (d == 0) {
            if (x + 1 >= g.nx) continue;
            w = u + 1;
        } else if (d == 1) {
            if (y + 1 >= g.ny) continue;
            w = u + g.nx;
        } else {
            if (z + 1 >= g.nz) continue;
            w = u + g.nxy;
        }
        // an inner vertex's word is (x, m) with m its descent minimum; any
        // other word belongs to a minimum. A minimum's word may be changing:
        // read it whole (tag-checked), or a torn (old s, new v) would look
        // like an inner vertex
        uint64_t ulo, uhi, wlo, whi;
        if (!wload(W, u, ulo, uhi) || !wload(W, w, wlo, whi)) {
            ok = false;
            continue;
        }
        const uint64_t mu = (ulo & kIdMask) == u ? (uhi & kIdMask) : u;
        const uint64_t mw = (wlo & kIdMask) == w ? (whi & kIdMask) : w;
        if (mu == mw) continue;
        const uint64_t S = before_w(f[u], u, f[w], w) ? w : u;
        ok &= M.merge(S, mu, mw);
    }
    if (!ok) raise_status(status, ST_TIMEOUT);
}

// ---------------------------------------------------------------- repair
// Representative (Algorithm 4) at level S: hop while the link's saddle is at
// or below S in the order; return the vertex where the walk stops. Concurrent
// repairs only move a word's target further along its own chain below the
// same saddle, so either half may be old or new.
__device__ __forceinline__ uint64_t w_rep(const uint64_t *W, const FieldW &f, uint64_t x, uint64_t S, float fS,
                                          uint32_t &steps)
{
    for (;;) {
        const uint64_t s = ld_rel(W + 2 * x) & kIdMask, v = ld_rel(W + 2 * x + 1) & kIdMask;
        if (s == x && v == x) return x;
        if (s != S && !before_w(f[s], s, fS, S)) return x;
        x = v;
        if (++steps > kChaseLimit) return x;
    }
}

__global__ void __launch_bounds__(kWThreads) k_w_repair(FieldW f, Geo g, uint64_t *W, uint32_t *status)
{
    if (*status) return;
    bool ok = true;
    for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < g.n; u += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t lo = ld_rel(W + 2 * u), hi = ld_rel(W + 2 * u + 1);
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
        if (r != v || lo != s || hi != v) {
            asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(W + 2 * u), "l"(s) : "memory");
            asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(W + 2 * u + 1), "l"(r) : "memory");
        }
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

// exclusive scan of the chunk counts into 64-bit offsets (one CTA)
__global__ void __launch_bounds__(1024) k_w_scan(const uint32_t *counts, uint64_t *offsets, uint64_t m,
                                                 uint64_t *meta, const uint32_t *status)
{
    if (block_skips(status)) return;
    __shared__ uint64_t part[1024];
    const uint64_t per = (m + 1023) / 1024;
    const uint64_t a = threadIdx.x * per, b = a + per < m ? a + per : m;
    uint64_t s = 0;
    for (uint64_t i = a; i < b; i++) s += counts[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const uint64_t v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint64_t run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (uint64_t i = a; i < b; i++) {
        offsets[i] = run;
        run += counts[i];
    }
    if (threadIdx.x == 1023) meta[0] = part[1023];
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
        const uint64_t su = W[2 * u], vu = W[2 * u + 1];
        uint64_t x = (su == u && vu != u) ? vu : u;
        for (uint64_t h = 0;; h++) {
            const uint64_t s = W[2 * x], v = W[2 * x + 1];
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
    const FieldW f{d_f, (flags & MT_SUPERLEVEL) ? -1.0f : 1.0f};
    if (cudaMemsetAsync(ws.status, 0, 768, s) != cudaSuccess) return MT_ERR_CUDA;
    {
        PhaseScope ps(kTile, s);
        k_w_init<<<grid_for(geo.n), kWThreads, 0, s>>>(f, geo, d_W, ws.status);
        for (int p = 0; p < kJumpPasses; p++)
            k_w_jump<<<grid_for(geo.n), kWThreads, 0, s>>>(geo, d_W, ws.jflag, p, ws.status);
        k_w_jump_check<<<1, 1, 0, s>>>(ws.jflag, ws.status);
        count_launch(2 + kJumpPasses);
    }
    {
        PhaseScope ps(kMerge, s);
        k_w_merge<<<grid_for(3 * geo.n), kWThreads, 0, s>>>(f, geo, d_W, ws.status);
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
