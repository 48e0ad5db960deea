// Kernels that build the triplet merge tree (Algorithm 1 of the paper):
//   k_tile     per tile, in shared memory: initialisation seeded with the
//              lowest lower neighbour, descent pointer jumping, Merge of the
//              in-tile edges, Repair
//   k_cross    Merge (Algorithm 3) of the edges between tiles, 64-bit CAS
//   k_repair   Repair (Algorithm 5) via Representative (Algorithm 4)
#include <cuda_runtime.h>

#include "mt_device.cuh"
#include "mt_internal.h"

namespace mt {

// ---------------------------------------------------------------- k_tile
//
// The initialisation loop and most of the edge loop of Algorithm 1, one
// brick ("tile") of the grid per CTA, entirely in shared memory.
//
// Algorithm 1 may merge the edges in any order. This kernel merges first the
// edges inside each tile: it loads the tile's values into shared memory
// (coalesced float4 rows), builds the triplet tree of the tile's own subgraph
// with the lock-free Merge (32-bit CAS on shared memory, local ids packed as
// (s << 16) | v), repairs it, and writes it out as global triplets. Local ids
// l = lx + TX * (ly + TY * lz) order the tile's vertices exactly as their
// global linear indices do, so ties break identically. Values are kept as
// 32-bit keys whose unsigned order is the float order (-0 and +0 share one
// key), so a vertex comparison is an integer comparison of (key, id).
//
// Within the tile the initial tree is seeded along steepest descent:
// T[l] = (l, lln(l)) with lln(l) the first vertex of l's closed in-tile
// neighbourhood (a normalised triplet of the graph of descent edges); pointer
// jumping then moves every inner vertex straight to the minimum its descent
// reaches, and an edge whose two ends reach the same minimum needs no merge.
//
// The merges themselves are organised for SIMT execution: the CTA first
// lists the edges that need a merge (task list in shared memory), then every
// lane pulls tasks dynamically and advances its merge by one climb step per
// iteration of a loop in which the whole warp stays converged, so lanes with
// short and long climbs do not serialise each other.
//
// What leaves the kernel is, for every vertex, its triplet in the subgraph
// induced by its tile: a valid normalised triplet tree of the full grid minus
// the edges between tiles, which k_cross merges next.
template <int LX, int LY, int LZ>
struct Tile {
    static constexpr int TX = 1 << LX, TY = 1 << LY, TZ = 1 << LZ;
    static constexpr int TV = TX * TY * TZ;
    static_assert(TV <= 16384, "tasks pack a local id and a direction into 16 bits");
    static_assert(TX % 4 == 0, "rows are loaded as float4");
    // shared memory: keys, triplets (4 B each) and up to 3 tasks (2 B each)
    static constexpr size_t kSmem = (size_t)TV * (4 + 4 + 6);
};

__device__ __forceinline__ uint32_t sm_pack(uint32_t s, uint32_t v) { return (s << 16) | v; }
__device__ __forceinline__ uint32_t sm_s(uint32_t w) { return w >> 16; }
__device__ __forceinline__ uint32_t sm_v(uint32_t w) { return w & 0xFFFFu; }

// Order-preserving 32-bit key of a float (+0 and -0 map to the same key).
__device__ __forceinline__ uint32_t order_key(float x)
{
    const uint32_t b = x == 0.0f ? 0u : __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
// (ka, a) before (kb, b)
__device__ __forceinline__ bool kbefore(uint32_t ka, uint32_t a, uint32_t kb, uint32_t b)
{
    return ka < kb || (ka == kb && a < b);
}

// Representative (Algorithm 4) in the tile's tree at level (kS, S).
// Every link leads to an earlier vertex, so a chain is shorter than the tile;
// a longer one can only come from a corrupted tree and clears ok.
template <int TV>
__device__ __forceinline__ uint32_t sm_rep(const uint32_t *T, const uint32_t *K, uint32_t x, uint32_t S,
                                           uint32_t kS, bool &ok)
{
    const volatile uint32_t *vT = T;
    for (uint32_t h = 0; h < (uint32_t)TV; h++) {
        const uint32_t w = vT[x];
        if (w == sm_pack(x, x)) return x;
        const uint32_t s = sm_s(w);
        if (s != S && !kbefore(K[s], s, kS, S)) return x;
        x = sm_v(w);
    }
    ok = false;
    return x;
}

template <int LX, int LY, int LZ, int NT>
__global__ void __launch_bounds__(NT, 2) k_tile(const float *__restrict__ f, uint64_t *__restrict__ W, uint32_t nx,
                                                uint32_t ny, uint32_t nz, uint32_t ntx, uint32_t nty, int vec,
                                                uint32_t *status)
{
    using TS = Tile<LX, LY, LZ>;
    constexpr int TX = TS::TX, TY = TS::TY, TZ = TS::TZ, TV = TS::TV;
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *K = smem;       // order keys
    uint32_t *T = smem + TV;  // triplets (s << 16) | v
    uint16_t *task = reinterpret_cast<uint16_t *>(smem + 2 * TV);
    __shared__ uint32_t s_ntask, s_next;

    const uint32_t lane = threadIdx.x & 31;
    const uint32_t tile = blockIdx.x;
    const uint32_t tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
    const uint32_t x0 = tx * TX, y0 = ty * TY, z0 = tz * TZ;
    const uint32_t wx = min((uint32_t)TX, nx - x0), wy = min((uint32_t)TY, ny - y0),
                   wz = min((uint32_t)TZ, nz - z0);
    const uint64_t nxy = (uint64_t)nx * ny;
    const uint64_t base = (uint64_t)z0 * nxy + (uint64_t)y0 * nx + x0;
    auto lxo = [](uint32_t l) { return l & (TX - 1); };
    auto lyo = [](uint32_t l) { return (l >> LX) & (TY - 1); };
    auto lzo = [](uint32_t l) { return l >> (LX + LY); };
    auto valid = [&](uint32_t l) { return lxo(l) < wx && lyo(l) < wy && lzo(l) < wz; };
    auto gid = [&](uint32_t l) {
        return (uint32_t)(base + (uint64_t)lzo(l) * nxy + (uint64_t)lyo(l) * nx + lxo(l));
    };
    if (threadIdx.x == 0) s_ntask = 0, s_next = 0;

    // 1. load the tile's values (rows of TX floats) as order keys
    bool bad = false;
    if (vec) {
        for (uint32_t q = threadIdx.x; q < TV / 4; q += NT) {
            const uint32_t l = 4 * q;
            if (lxo(l) < wx && lyo(l) < wy && lzo(l) < wz) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(f + gid(l)));
                bad |= !isfinite(v.x) | !isfinite(v.y) | !isfinite(v.z) | !isfinite(v.w);
                *reinterpret_cast<uint4 *>(K + l) = make_uint4(order_key(v.x), order_key(v.y), order_key(v.z),
                                                              order_key(v.w));
            }
        }
    } else {
        for (uint32_t l = threadIdx.x; l < TV; l += NT) {
            if (valid(l)) {
                const float v = __ldg(f + gid(l));
                bad |= !isfinite(v);
                K[l] = order_key(v);
            }
        }
    }
    if (bad) raise_status(status, ST_NONFINITE);
    __syncthreads();

    // 2. seed: T[l] = (l, first vertex of the closed in-tile neighbourhood)
    for (uint32_t l = threadIdx.x; l < TV; l += NT) {
        if (!valid(l)) continue;
        const uint32_t lx = lxo(l), ly = lyo(l), lz = lzo(l);
        uint32_t b = l, kb = K[l];
        // candidates in ascending local index order: an earlier id wins ties,
        // so an earlier candidate replaces b only if strictly lower
        if (lz > 0 && K[l - TX * TY] <= kb) b = l - TX * TY, kb = K[b];
        if (ly > 0 && K[l - TX] <= kb && (K[l - TX] < kb || l - TX < b)) b = l - TX, kb = K[b];
        if (lx > 0 && K[l - 1] <= kb && (K[l - 1] < kb || l - 1 < b)) b = l - 1, kb = K[b];
        if (lx + 1 < wx && K[l + 1] < kb) b = l + 1, kb = K[b];
        if (ly + 1 < wy && K[l + TX] < kb) b = l + TX, kb = K[b];
        if (lz + 1 < wz && K[l + TX * TY] < kb) b = l + TX * TY, kb = K[b];
        T[l] = sm_pack(l, b);
    }
    __syncthreads();

    // 3. pointer jumping along the descent links (concurrent jumps only
    //    shorten chains, so racing readers stay correct)
    {
        volatile uint32_t *vT = T;
        for (uint32_t l = threadIdx.x; l < TV; l += NT) {
            if (!valid(l)) continue;
            const uint32_t w = vT[l];
            if (sm_v(w) == l) continue;  // a minimum
            uint32_t x = sm_v(w);
            for (uint32_t h = 0; h < (uint32_t)TV; h++) {
                const uint32_t wx_ = vT[x];
                if (sm_v(wx_) == x) break;
                x = sm_v(wx_);
            }
            if (x != sm_v(w)) vT[l] = sm_pack(l, x);
        }
    }
    __syncthreads();

    // 4a. list the in-tile edges to the +x, +y, +z neighbours whose ends
    //     descend to different minima (warp-aggregated appends)
    for (uint32_t l0 = 0; l0 < TV; l0 += NT) {
        const uint32_t l = l0 + threadIdx.x;
        uint32_t mask = 0;
        if (valid(l)) {
            const uint32_t dl = sm_v(T[l]);  // descent minimum (l itself for a minimum)
            const uint32_t lx = lxo(l), ly = lyo(l), lz = lzo(l);
            if (lx + 1 < wx && sm_v(T[l + 1]) != dl) mask |= 1;
            if (ly + 1 < wy && sm_v(T[l + TX]) != dl) mask |= 2;
            if (lz + 1 < wz && sm_v(T[l + TX * TY]) != dl) mask |= 4;
        }
        const uint32_t cnt = __popc(mask);
        uint32_t incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
        uint32_t wbase = 0;
        if (lane == 31 && tot) wbase = atomicAdd(&s_ntask, tot);
        wbase = __shfl_sync(0xffffffffu, wbase, 31);
        uint32_t pos = wbase + incl - cnt;
        for (int d = 0; d < 3; d++)
            if (mask & (1u << d)) task[pos++] = (uint16_t)((l << 2) | d);
    }
    __syncthreads();

    // 4b. run the merges (Algorithm 3), one climb step per converged
    //     iteration; idle lanes fetch the next task
    {
        const uint32_t ntask = s_ntask;
        const volatile uint32_t *vT = T;
        bool busy = false, cu = false, cv = false, ok = true, drained = false;
        uint32_t S = 0, kS = 0, u = 0, v = 0, Tu = 0, Tv = 0;
        uint32_t steps = 0;
        for (;;) {
            const uint32_t idle = __ballot_sync(0xffffffffu, !busy);
            if (idle && !drained) {
                uint32_t tb = 0;
                const uint32_t leader = __ffs(idle) - 1;
                if (lane == leader) tb = atomicAdd(&s_next, __popc(idle));
                tb = __shfl_sync(0xffffffffu, tb, leader);
                drained = tb + __popc(idle) >= ntask;
                if (!busy) {
                    const uint32_t t = tb + __popc(idle & ((1u << lane) - 1u));
                    if (t < ntask) {
                        const uint32_t code = task[t];
                        const uint32_t l = code >> 2, d = code & 3;
                        const uint32_t w = l + (d == 0 ? 1u : d == 1 ? (uint32_t)TX : (uint32_t)(TX * TY));
                        const uint32_t kl = K[l], kw = K[w];
                        if (kbefore(kw, w, kl, l)) S = l, kS = kl;
                        else S = w, kS = kw;
                        // descent minimum: an inner vertex's target; a
                        // minimum (whose entry other merges may have linked
                        // already, s != itself) stands for itself
                        const uint32_t Tl = vT[l], Tw = vT[w];
                        u = sm_s(Tl) == l ? sm_v(Tl) : l;
                        v = sm_s(Tw) == w ? sm_v(Tw) : w;
                        busy = cu = cv = true;
                        steps = 0;
                    }
                }
            }
            if (!__any_sync(0xffffffffu, busy)) break;
            if (busy) {
                // one step of each unfinished climb (links whose saddle is at
                // or below S are followed; a root stops the climb)
                if (cu) {
                    Tu = vT[u];
                    const uint32_t s = sm_s(Tu);
                    if (Tu == sm_pack(u, u) || (s != S && !kbefore(K[s], s, kS, S))) cu = false;
                    else u = sm_v(Tu);
                }
                if (cv) {
                    Tv = vT[v];
                    const uint32_t s = sm_s(Tv);
                    if (Tv == sm_pack(v, v) || (s != S && !kbefore(K[s], s, kS, S))) cv = false;
                    else v = sm_v(Tv);
                }
                if (++steps > kMergeStepLimit) {
                    ok = false;
                    busy = false;
                } else if (!cu && !cv) {
                    if (u == v) {
                        busy = false;
                    } else {
                        if (kbefore(K[v], v, K[u], u)) {
                            const uint32_t x = u;
                            u = v;
                            v = x;
                            const uint32_t y = Tu;
                            Tu = Tv;
                            Tv = y;
                        }
                        if (atomicCAS(T + v, Tv, sm_pack(S, u)) == Tv) {
                            if (Tv == sm_pack(v, v)) {
                                busy = false;
                            } else {  // re-insert the displaced link
                                S = sm_s(Tv);
                                kS = K[S];
                                v = sm_v(Tv);
                            }
                        }
                        cu = cv = busy;
                    }
                }
            }
        }
        if (!ok) raise_status(status, ST_TIMEOUT);
    }
    __syncthreads();

    // 5. repair (Algorithm 5): branch minima first, then inner vertices
    bool rep_ok = true;
    for (uint32_t l = threadIdx.x; l < TV; l += NT) {
        if (!valid(l)) continue;
        const uint32_t w = T[l];
        const uint32_t s = sm_s(w);
        if (s == l) continue;
        const uint32_t r = sm_rep<TV>(T, K, sm_v(w), s, K[s], rep_ok);
        if (r != sm_v(w)) T[l] = sm_pack(s, r);
    }
    __syncthreads();
    for (uint32_t l = threadIdx.x; l < TV; l += NT) {
        if (!valid(l)) continue;
        const uint32_t w = T[l];
        if (sm_s(w) != l || sm_v(w) == l) continue;
        const uint32_t r = sm_rep<TV>(T, K, sm_v(w), l, K[l], rep_ok);
        if (r != sm_v(w)) T[l] = sm_pack(l, r);
    }
    if (!rep_ok) raise_status(status, ST_TIMEOUT);
    __syncthreads();

    // 6. write the tile's triplets with global ids (coalesced rows)
    if (vec) {
        for (uint32_t q = threadIdx.x; q < TV / 2; q += NT) {
            const uint32_t l = 2 * q;
            if (!valid(l)) continue;
            const uint32_t T0 = T[l], T1 = T[l + 1];
            *reinterpret_cast<ulonglong2 *>(W + gid(l)) = make_ulonglong2(
                tri_pack(gid(sm_s(T0)), gid(sm_v(T0))), tri_pack(gid(sm_s(T1)), gid(sm_v(T1))));
        }
    } else {
        for (uint32_t l = threadIdx.x; l < TV; l += NT) {
            if (!valid(l)) continue;
            const uint32_t w = T[l];
            W[gid(l)] = tri_pack(gid(sm_s(w)), gid(sm_v(w)));
        }
    }
}

// ---------------------------------------------------------------- k_cross
//
// The rest of the edge loop of Algorithm 1: the edges between neighbouring
// tiles, merged with 64-bit CAS on the global triplets (Algorithms 2, 3).
// CTA t takes the edges from tile t to its +x, +y, +z neighbour tiles, so
// the climbs of one CTA stay mostly within a few tiles' entries (L2 reuse).
// A merge for edge (a, b) at level S = the later of a, b starts at a and b
// themselves; their tile triplets lead to the tile-local deepest vertices.
template <int LX, int LY, int LZ>
__global__ void __launch_bounds__(256) k_cross(uint64_t *W, const float *__restrict__ f, uint32_t nx, uint32_t ny,
                                               uint32_t nz, uint32_t ntx, uint32_t nty, uint32_t *status)
{
    if (*status) return;
    using TS = Tile<LX, LY, LZ>;
    constexpr uint32_t TX = TS::TX, TY = TS::TY, TZ = TS::TZ;
    const uint32_t tile = blockIdx.x;
    const uint32_t tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
    const uint32_t x0 = tx * TX, y0 = ty * TY, z0 = tz * TZ;
    const uint32_t wx = min(TX, nx - x0), wy = min(TY, ny - y0), wz = min(TZ, nz - z0);
    const uint32_t nxy = nx * ny;
    const uint32_t base = z0 * nxy + y0 * nx + x0;
    const uint32_t cx = (x0 + TX < nx) ? wy * wz : 0;
    const uint32_t cy = (y0 + TY < ny) ? wx * wz : 0;
    const uint32_t cz = (z0 + TZ < nz) ? wx * wy : 0;
    bool ok = true;
    for (uint32_t e = threadIdx.x; e < cx + cy + cz; e += blockDim.x) {
        uint32_t a, b;
        if (e < cx) {
            a = base + (e / wy) * nxy + (e % wy) * nx + (TX - 1);
            b = a + 1;
        } else if (e < cx + cy) {
            const uint32_t k = e - cx;
            a = base + (k / wx) * nxy + (TY - 1) * nx + (k % wx);
            b = a + nx;
        } else {
            const uint32_t k = e - cx - cy;
            a = base + (TZ - 1) * nxy + (k / wx) * nx + (k % wx);
            b = a + nxy;
        }
        const uint32_t S = before(__ldg(f + b), b, __ldg(f + a), a) ? a : b;
        ok &= merge(W, f, S, a, b);
    }
    if (!ok) raise_status(status, ST_TIMEOUT);
}

// --------------------------------------------------------------- k_repair
//
// Repair (Algorithm 5): T[u] = (s, Representative(u, s)) restores
// minimality. Level comparisons use the vertex order, not values alone:
// with tied values a saddle s' equal in value to s but after it in the order
// is not yet part of the sublevel set at s. Concurrent repairs only replace a
// target by one further along the same chain below the same level, so a
// chase that reads a freshly repaired entry reaches the same answer sooner.
// mode 0 repairs branch minima (s != u), mode 1 the inner vertices
// (s == u != v); running mode 0 first leaves the chains of mode 1 minimal.
// Because every rewrite keeps a link on the same chain, a stale cached copy of
// an entry is still a valid (longer) way to the same answer, so the chases
// use ordinary L1-cached loads.
__global__ void __launch_bounds__(256) k_repair(uint64_t *W, const float *__restrict__ f, uint64_t n, int mode,
                                                uint32_t *status)
{
    if (*status) return;
    for (uint64_t uu = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; uu < n;
         uu += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t u = (uint32_t)uu;
        const uint64_t T = W[u];
        const uint32_t s = tri_s(T), t = tri_v(T);
        if (mode == 0 ? (s == u) : (s != u || t == u)) continue;
        uint32_t steps = 0;
        const uint32_t r = representative_cached(W, f, t, s, __ldg(f + s), steps);
        if (steps > kChaseLimit) {
            raise_status(status, ST_TIMEOUT);
            continue;
        }
        if (r != t) st_tri(W + u, tri_pack(s, r));
    }
}

// ------------------------------------------------------------ host side

static int grid_for(uint64_t work, int threads)
{
    const uint64_t want = (work + threads - 1) / threads;
    const uint64_t cap = (uint64_t)device_sms() * 8;  // 8 resident 256-thread CTAs per SM
    return (int)(want < cap ? (want ? want : 1) : cap);
}

// Tile shape 32 x 16 x 16: 8192 vertices, 112 KiB of shared memory, two
// CTAs of 1024 threads per SM.
constexpr int kLX = 5, kLY = 4, kLZ = 4, kTileThreads = 1024;

cudaError_t launch_build(const float *f, uint64_t *W, uint32_t nx, uint32_t ny, uint32_t nz, Workspace &ws,
                         cudaStream_t st)
{
    using TS = Tile<kLX, kLY, kLZ>;
    const uint64_t n = (uint64_t)nx * ny * nz;
    const int vec = (nx % 4 == 0) && ((uintptr_t)f % 16 == 0) && ((uintptr_t)W % 16 == 0);
    const uint32_t ntx = (nx + TS::TX - 1) / TS::TX, nty = (ny + TS::TY - 1) / TS::TY,
                   ntz = (nz + TS::TZ - 1) / TS::TZ;
    const uint64_t ntiles = (uint64_t)ntx * nty * ntz;
    const size_t smem = TS::kSmem;
    cudaError_t e;
    static bool attr_done = false;
    if (!attr_done) {
        e = cudaFuncSetAttribute(k_tile<kLX, kLY, kLZ, kTileThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_tile<kLX, kLY, kLZ, kTileThreads>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    {
        PhaseScope ps(kTile, st);
        k_tile<kLX, kLY, kLZ, kTileThreads><<<(unsigned)ntiles, kTileThreads, smem, st>>>(f, W, nx, ny, nz, ntx,
                                                                                         nty, vec, ws.status);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        PhaseScope ps(kMerge, st);
        k_cross<kLX, kLY, kLZ><<<(unsigned)ntiles, 256, 0, st>>>(W, f, nx, ny, nz, ntx, nty, ws.status);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    PhaseScope ps(kRepair, st);
    k_repair<<<grid_for(n, 256), 256, 0, st>>>(W, f, n, 0, ws.status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_repair<<<grid_for(n, 256), 256, 0, st>>>(W, f, n, 1, ws.status);
    count_launch(2);
    return cudaGetLastError();
}

}  // namespace mt
