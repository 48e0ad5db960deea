// Device-side building blocks of the triplet merge tree (sm_103a).
//
// Triplet word:  W[u] = (s << 32) | v  encodes the triplet (u, s, v)
// (Section 2.1; one 64-bit word per vertex as in Section 3.2, so that a single
// 64-bit compare-and-swap updates the pair).
// Order:         a < b  <=>  f[a] < f[b] || (f[a] == f[b] && a < b).
#pragma once
#include <cstdint>

namespace mt {

// Status bits kept in the first word of the workspace.
enum : uint32_t {
    ST_NONFINITE = 1u,
    ST_TIMEOUT = 2u,
    ST_CAPACITY = 4u,
    ST_CORRUPT = 8u,  // a triplet array given by the caller holds an id >= n
};

// Table sizes of the shared-memory hashes and lists. Each table has a path
// for when it is full (merge in place, repair from an overflow bitmap, chase
// the global chain); the defaults keep those paths rare. A library built with
// MT_STRESS_TABLES shrinks the tables so that the tests reach every such
// path; its results are the same.
#ifdef MT_STRESS_TABLES
constexpr uint32_t kTileHashProbes = 1;   // k_tile: probes before merging in place
constexpr uint32_t kRepairShrink = 64;    // k_repair: hash, copies and minima list 64x smaller
constexpr uint32_t kLabelHashLog = 6;     // k_labels: 64 chain starts per brick
#else
constexpr uint32_t kTileHashProbes = 16;
constexpr uint32_t kRepairShrink = 1;
constexpr uint32_t kLabelHashLog = 12;    // 4096 chain starts per brick
#endif

// Limits of the bounded device loops. A merge that needs more steps than this
// gives up and raises ST_TIMEOUT instead of spinning.
constexpr uint32_t kMergeStepLimit = 1u << 24;
constexpr uint32_t kChaseLimit = 1u << 24;

__device__ __forceinline__ uint32_t tri_s(uint64_t w) { return (uint32_t)(w >> 32); }
__device__ __forceinline__ uint32_t tri_v(uint64_t w) { return (uint32_t)w; }
__device__ __forceinline__ uint64_t tri_pack(uint32_t s, uint32_t v) { return ((uint64_t)s << 32) | v; }

// a before b in the total order (value, index)
__device__ __forceinline__ bool before(float fa, uint32_t a, float fb, uint32_t b)
{
    return fa < fb || (fa == fb && a < b);
}

// Loads of triplet words that other threads may be updating concurrently:
// relaxed, device scope, so that they are not served from a stale L1 line.
__device__ __forceinline__ uint64_t ld_tri(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_tri(uint64_t *p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t cas_tri(uint64_t *p, uint64_t expect, uint64_t want)
{
    return atomicCAS(reinterpret_cast<unsigned long long *>(p), (unsigned long long)expect,
                     (unsigned long long)want);
}

__device__ __forceinline__ void raise_status(uint32_t *status, uint32_t bit) { atomicOr(status, bit); }

// Whether a CTA skips its work because an earlier error is recorded. The
// status word may be raised by another CTA at any moment, so one thread reads
// it and every thread gets that one answer: kernels with barriers must leave
// (or stay) as a whole block.
__device__ __forceinline__ bool block_skips(const uint32_t *status)
{
    return __syncthreads_or(threadIdx.x == 0 && *(const volatile uint32_t *)status != 0) != 0;
}

// The values as the order sees them: f itself (sublevel sets), or -f (sg =
// -1) for the tree of the superlevel sets, the split tree. Multiplying by -1
// is exact, and -0 still equals +0.
struct Field {
    const float *f;
    float sg;
    __device__ __forceinline__ float operator[](uint32_t i) const { return sg * __ldg(f + i); }
};

// Climbs (Algorithm 3): follow the triplet links from a vertex while the
// link's saddle is at or below level S (vertex order), i.e. walk to the
// deepest vertex that the current tree connects to it below S. A root word
// (x, x) always stops a walk (the paper's pseudocode has no guard for it).
// Both climbs of a merge side by side, so that their loads overlap: each
// round reads, for every walk still going, its saddle's value and (before the
// level test) its next vertex's word.
__device__ __forceinline__ void climb2(const uint64_t *W, const Field f, uint32_t &u, uint32_t &v, uint32_t S,
                                       float fS, uint64_t &Tu, uint64_t &Tv, uint32_t &steps)
{
    Tu = ld_tri(W + u);
    Tv = ld_tri(W + v);
    bool du = false, dv = false;
    for (;;) {
        const uint32_t su = tri_s(Tu), tu = tri_v(Tu), sv = tri_s(Tv), tv = tri_v(Tv);
        du = du || (su == u && tu == u);
        dv = dv || (sv == v && tv == v);
        float fsu = 0.0f, fsv = 0.0f;
        uint64_t Tnu = 0, Tnv = 0;
        if (!du) fsu = f[su], Tnu = ld_tri(W + tu);
        if (!dv) fsv = f[sv], Tnv = ld_tri(W + tv);
        du = du || (su != S && !before(fsu, su, fS, S));
        dv = dv || (sv != S && !before(fsv, sv, fS, S));
        if (du && dv) return;
        if (!du) u = tu, Tu = Tnu;
        if (!dv) v = tv, Tv = Tnv;
        if (++steps > kMergeStepLimit) return;
    }
}

// Algorithm 3 (Merge), lock-free: make a and b connected at level S in the
// triplet forest, given that they are connected below S in the graph.
//   1. climb a and b to their deepest vertices u, v below S;
//   2. if they coincide the edge adds nothing;
//   3. otherwise order them so that u comes first and swing v's link to
//      (S, u) with one 64-bit CAS (Algorithm 2);
//   4. the link that v held before, (sv, tv), is not lost: if v was not a
//      root, continue by merging u and tv at level sv. (A displaced root
//      carries no link, so the merge ends there.)
//   5. if the CAS fails another thread moved v first: climb again.
// Returns false if the step budget ran out.
__device__ __forceinline__ bool merge(uint64_t *W, const Field f, uint32_t S, uint32_t a, uint32_t b)
{
    float fS = f[S];
    uint32_t u = a, v = b;
    uint32_t steps = 0;
    for (;;) {
        uint64_t Tu, Tv;
        climb2(W, f, u, v, S, fS, Tu, Tv, steps);
        if (++steps > kMergeStepLimit) return false;
        if (u == v) return true;
        if (before(f[v], v, f[u], u)) {
            uint32_t tx = u;
            u = v;
            v = tx;
            uint64_t tT = Tu;
            Tu = Tv;
            Tv = tT;
        }
        const uint64_t old = cas_tri(W + v, Tv, tri_pack(S, u));
        if (old == Tv) {
            const uint32_t sv = tri_s(Tv), tv = tri_v(Tv);
            if (sv == v && tv == v) return true;  // displaced a root
            S = sv;
            fS = f[sv];
            v = tv;
        }
    }
}

// Representative (Algorithm 4) of x at level S given as a vertex: the deepest
// vertex of x's component below S. Hops while the link's saddle s' satisfies
// s' <= S in the vertex order and returns the vertex where it stops (the
// printed algorithm returns one hop further; the vertex itself is the one
// the definition asks for). Ordinary (L1-cacheable) loads: it serves passes
// in which the entries only ever move further along their own chains
// (repair), where a stale copy still leads to the same representative. The
// triplet of the next vertex is loaded together with the value of the
// current saddle, before the level test decides whether it is needed, so that
// a hop costs one memory latency instead of two (the extra load reads a valid
// entry either way).
__device__ __forceinline__ uint32_t representative_cached(const uint64_t *W, const Field f, uint32_t x, uint32_t S,
                                                          float fS, uint32_t &steps)
{
    uint64_t T = W[x];
    for (;;) {
        const uint32_t s = tri_s(T), t = tri_v(T);
        if (s == x && t == x) return x;
        const float fs = f[s];
        const uint64_t Tn = W[t];
        if (s != S && !before(fs, s, fS, S)) return x;
        x = t;
        T = Tn;
        if (++steps > kChaseLimit) return x;
    }
}

}  // namespace mt
