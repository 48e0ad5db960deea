// Kernels that build the triplet merge tree (Algorithm 1 of the paper):
//   k_tile     per tile, in shared memory: initialisation seeded with the
//              lowest lower neighbour, descent pointer jumping, Merge of the
//              in-tile edges, Repair
//   k_cross    Merge (Algorithm 3) of the edges between tiles, 64-bit CAS
//   k_repair   Repair (Algorithm 5) via Representative (Algorithm 4); in
//              mt_build_components also the components of G_t
#include <cuda_runtime.h>

#include <type_traits>

#include "mt_device.cuh"
#include "mt_fields.cuh"
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
// Seed. T[l] = (l, lln(l)), lln(l) the first vertex of l's closed in-tile
// neighbourhood (a normalised triplet of the graph of steepest-descent
// edges); pointer jumping then moves every inner vertex straight to the
// minimum its descent reaches. An edge whose ends reach the same minimum
// needs no merge.
//
// Level buckets and shortcuts. The remaining edges are merged in NB rounds
// by the level of their upper end S (NB buckets of about equal size, cut from
// a histogram of the tile's keys); within a round the order is free, as
// Algorithm 1 allows. SC[m] is a shortcut for minimum m: the vertex m's climb
// reaches through the links whose saddle lies in buckets before the current
// one, i.e. the deepest vertex of m's component below the round. Those links
// do not change during a round (a merge at level S only displaces links above
// S), so a shortcut is computed on first use in a round and stored with the
// round number in its top bits. An edge (S, a, c) starts its climbs at SC[a]
// and SC[c] (both joined to a, c below S), and when they coincide the ends are
// already connected below S and the edge is settled by two shared-memory
// loads, as about nine edges in ten are on these fields. The others are
// collected and merged together once the bucket's scan is done, so that the
// lanes of a warp run their merges side by side instead of one after another.
// They are collected in a shared-memory hash keyed by the pair of shortcuts
// that keeps, per pair, only the edge with the earliest upper end: once that
// one is merged, the two components are joined below the level of every
// other edge of the pair, which Merge would then find connected and skip. On
// these fields about two collected edges in five repeat a pair.
//
// Repair. Right after round b no later merge can change a component below
// the levels of bucket b, so every inner vertex l of bucket b gets its final
// tile triplet (l, deepest vertex below l) by a short climb from its
// minimum's shortcut (Algorithms 4 and 5). Branch minima are repaired at the
// end.
//
// What leaves the kernel is, for every vertex, its triplet in the subgraph
// induced by its tile: a valid normalised triplet tree of the full grid minus
// the edges between tiles, which k_cross merges next.
constexpr int log2i(int x) { return x <= 1 ? 0 : 1 + log2i(x / 2); }

template <int LX, int LY, int LZ, int NT = 512>
struct Tile {
    static constexpr int TX = 1 << LX, TY = 1 << LY, TZ = 1 << LZ;
    static constexpr int TV = TX * TY * TZ;
    static_assert(TV <= 65536, "local ids are 16-bit");
    static_assert(TX % 4 == 0, "rows are loaded as float4");
    static constexpr int kBins = NT;     // key histogram, one bin per thread
    static constexpr int kQueue = 2048 * TV / 8192 > NT ? 2048 * TV / 8192 : NT;  // 32-bit words of the edge hash
    static constexpr int kHashLog = log2i(kQueue / 3);                            // slots: 32-bit pair + 64-bit level
    static constexpr int kHash = 1 << kHashLog;
    static_assert(kHash * 12 <= kQueue * 4, "hash fits its buffer");
    // shared memory: keys + triplets (4 B each), shortcuts + bucket-sorted
    // vertex list (2 B each), edge hash (aliased by the key histogram)
    static constexpr size_t kSmem = (size_t)TV * (4 + 4 + 2 + 2) + (size_t)kQueue * 4;
    static_assert(kQueue >= kBins, "the histogram lives in the hash buffer");
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

// Climb (Algorithm 3 / 4) in the tile's tree from x through links whose
// saddle is at or below (kS, S); a root stops it. Chains lead to ever earlier
// vertices, so a walk longer than the tile means a corrupted tree (ok=false).
// The next vertex's triplet is read together with the saddle's key, before
// the test that decides whether it is needed (indices are masked to the
// tile, so a read that turns out unneeded stays in bounds).
template <int TV>
__device__ __forceinline__ uint32_t sm_climb(const uint32_t *T, const uint32_t *K, uint32_t x, uint32_t S,
                                             uint32_t kS, uint32_t &w, bool &ok)
{
    const volatile uint32_t *vT = T;
    uint32_t wx = vT[x];
    for (uint32_t h = 0; h < (uint32_t)TV; h++) {
        const uint32_t s = sm_s(wx), nx = sm_v(wx);
        const uint32_t ks = K[s & (TV - 1)];
        const uint32_t wn = vT[nx & (TV - 1)];
        if (wx == sm_pack(x, x) || (s != S && !kbefore(ks, s, kS, S))) {
            w = wx;
            return x;
        }
        x = nx;
        wx = wn;
    }
    ok = false;
    w = wx;
    return x;
}

// Both climbs of a merge side by side, so that their reads overlap.
template <int TV>
__device__ __forceinline__ void sm_climb2(const uint32_t *T, const uint32_t *K, uint32_t &u, uint32_t &v,
                                          uint32_t S, uint32_t kS, uint32_t &wu, uint32_t &wv, bool &ok)
{
    const volatile uint32_t *vT = T;
    wu = vT[u], wv = vT[v];
    bool du = false, dv = false;
    for (uint32_t h = 0; h < 2u * TV; h++) {
        const uint32_t su = sm_s(wu), nu = sm_v(wu), sv = sm_s(wv), nv = sm_v(wv);
        const uint32_t ku = K[su & (TV - 1)], kv = K[sv & (TV - 1)];
        const uint32_t wnu = vT[nu & (TV - 1)], wnv = vT[nv & (TV - 1)];
        du = du || wu == sm_pack(u, u) || (su != S && !kbefore(ku, su, kS, S));
        dv = dv || wv == sm_pack(v, v) || (sv != S && !kbefore(kv, sv, kS, S));
        if (du && dv) return;
        if (!du) u = nu, wu = wnu;
        if (!dv) v = nv, wv = wnv;
    }
    ok = false;
}

// Merge (Algorithm 3) on the tile's shared-memory tree, lock-free with 32-bit
// CAS (Algorithm 2): climb a and c to their deepest vertices below S; if they
// differ, link the later one under the earlier at S and re-insert the link
// it held before (a displaced root carries none); on a failed CAS climb again.
template <int TV>
__device__ __forceinline__ void sm_merge(uint32_t *T, const uint32_t *K, uint32_t S, uint32_t kS, uint32_t a,
                                         uint32_t c, bool &ok)
{
    uint32_t u = a, v = c;
    for (uint32_t it = 0; it < kMergeStepLimit; it++) {
        uint32_t Tu, Tv;
        sm_climb2<TV>(T, K, u, v, S, kS, Tu, Tv, ok);
        if (!ok || u == v) return;
        if (kbefore(K[v], v, K[u], u)) {
            const uint32_t x = u;
            u = v;
            v = x;
            const uint32_t y = Tu;
            Tu = Tv;
            Tv = y;
        }
        if (atomicCAS(T + v, Tv, sm_pack(S, u)) == Tv) {
            if (Tv == sm_pack(v, v)) return;
            S = sm_s(Tv);
            kS = K[S];
            v = sm_v(Tv);
        }
    }
    ok = false;
}

// WIDE: the triplets leave the tile as 128-bit words of two 64-bit ids
// (W[2u] = s, W[2u + 1] = v) for grids of 2^32 vertices and more; the work
// inside the tile, on 16-bit local ids, is the same, and no face buffer is
// written (the wide path merges the edges between tiles from their ends).
template <int LX, int LY, int LZ, int NT, int NB, bool FULL, bool WIDE = false>
__device__ __forceinline__ void tile_body(const FieldDesc &fd, uint32_t tile, uint32_t *status)
{
    using Id = typename std::conditional<WIDE, uint64_t, uint32_t>::type;
    const float *__restrict__ f = fd.f;
    const float sg = fd.sg;
    uint64_t *__restrict__ W = fd.W;
    const uint32_t nx = fd.nx, ny = fd.ny, nz = fd.nz, ntx = fd.ntx, nty = fd.nty;
    const bool vec = (nx % 4 == 0) && ((uintptr_t)f % 16 == 0) && ((uintptr_t)W % 16 == 0);
    using TS = Tile<LX, LY, LZ, NT>;
    constexpr int TX = TS::TX, TY = TS::TY, TZ = TS::TZ, TV = TS::TV, BINS = TS::kBins, HS = TS::kHash, HLOG = TS::kHashLog;
    constexpr uint32_t IDB = LX + LY + LZ;  // bits of a local id
    constexpr uint32_t IDM = (1u << IDB) - 1u;
    static_assert(NT >= BINS, "one histogram bin per thread");
    static_assert(IDB + 3 <= 16 && NB <= 8, "a shortcut packs a local id and a round number into 16 bits");
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *K = smem;                                           // order keys
    uint32_t *T = smem + TV;                                      // triplets (s << 16) | v
    uint16_t *SC = reinterpret_cast<uint16_t *>(smem + 2 * TV);   // shortcuts (round << IDB) | vertex
    uint16_t *vlist = SC + TV;                                    // vertices sorted by bucket
    // edges to merge in the current round, one per pair of shortcuts:
    // hkey = (lo << IDB) | hi, hlev = (key << 32) | S of the earliest upper end
    unsigned long long *hlev = reinterpret_cast<unsigned long long *>(vlist + TV);
    uint32_t *hkey = reinterpret_cast<uint32_t *>(hlev + HS);
    uint32_t *hist = reinterpret_cast<uint32_t *>(hlev);          // key histogram (before the rounds)
    __shared__ uint8_t s_bmap[BINS];                              // histogram bin -> bucket
    __shared__ uint32_t s_nvalid, s_warp[NT / 32], s_wmin[NT / 32], s_wmax[NT / 32];
    __shared__ uint32_t s_boff[NB + 2], s_bcur[NB + 1], s_thr[NB];

    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
    const uint32_t x0 = tx * TX, y0 = ty * TY, z0 = tz * TZ;
    // a FULL tile lies inside the grid: its extents are the tile's
    const uint32_t wx = FULL ? (uint32_t)TX : min((uint32_t)TX, nx - x0),
                   wy = FULL ? (uint32_t)TY : min((uint32_t)TY, ny - y0),
                   wz = FULL ? (uint32_t)TZ : min((uint32_t)TZ, nz - z0);
    const Id nxy = (Id)nx * ny;  // n < 2^32 unless WIDE, so every id fits an Id
    const Id base = (Id)z0 * nxy + (Id)y0 * nx + x0;
    auto lxo = [](uint32_t l) { return l & (TX - 1); };
    auto lyo = [](uint32_t l) { return (l >> LX) & (TY - 1); };
    auto lzo = [](uint32_t l) { return l >> (LX + LY); };
    auto valid = [&](uint32_t l) { return FULL || (lxo(l) < wx && lyo(l) < wy && lzo(l) < wz); };
    auto gid = [&](uint32_t l) -> Id { return base + (Id)lzo(l) * nxy + (Id)lyo(l) * nx + lxo(l); };
    // (the barrier after the loads orders these writes before their uses)
    if (threadIdx.x == 0) s_nvalid = wx * wy * wz;
    if (threadIdx.x <= NB) s_bcur[threadIdx.x] = 0;
    for (uint32_t i = threadIdx.x; i < (uint32_t)BINS; i += NT) hist[i] = 0;

    // 1. load the tile's values (rows of TX floats) as order keys
    bool bad = false;
    uint32_t kmin = 0xFFFFFFFFu, kmax = 0;
    if (vec) {
        for (uint32_t q = threadIdx.x; q < TV / 4; q += NT) {
            const uint32_t l = 4 * q;
            if (valid(l)) {
                float4 v = __ldg(reinterpret_cast<const float4 *>(f + gid(l)));
                v.x *= sg, v.y *= sg, v.z *= sg, v.w *= sg;
                bad |= !isfinite(v.x) | !isfinite(v.y) | !isfinite(v.z) | !isfinite(v.w);
                const uint4 k = make_uint4(order_key(v.x), order_key(v.y), order_key(v.z), order_key(v.w));
                kmin = min(kmin, min(min(k.x, k.y), min(k.z, k.w)));
                kmax = max(kmax, max(max(k.x, k.y), max(k.z, k.w)));
                *reinterpret_cast<uint4 *>(K + l) = k;
            }
        }
    } else {
        for (uint32_t l = threadIdx.x; l < TV; l += NT) {
            if (valid(l)) {
                const float v = sg * __ldg(f + gid(l));
                bad |= !isfinite(v);
                const uint32_t k = order_key(v);
                kmin = min(kmin, k);
                kmax = max(kmax, k);
                K[l] = k;
            }
        }
    }
    if (bad) raise_status(status, ST_NONFINITE);
    for (int o = 16; o > 0; o >>= 1) {
        kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
        kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    }
    if (lane == 0) s_wmin[warp] = kmin, s_wmax[warp] = kmax;
    __syncthreads();
    kmin = lane < NT / 32 ? s_wmin[lane] : 0xFFFFFFFFu;
    kmax = lane < NT / 32 ? s_wmax[lane] : 0u;
    for (int o = 16; o > 0; o >>= 1) {
        kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
        kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    }

    // Spare bits of a triplet (ids take IDB of each 16-bit half) carry a
    // mask of neighbour directions d (-x, -y, -z, +x, +y, +z): from the seed
    // to step 4 the lower neighbours of the vertex, from step 4 on (inner
    // vertices only) its cross mask: the lower neighbours that descend to
    // another minimum. Only those edges can join two components; the scan of
    // the vertex's level bucket reads them from here. The bucket repair of
    // the vertex rewrites its triplet and so clears the bits; minima never
    // carry any (a minimum has no lower neighbour).
    auto tid_s = [](uint32_t w) { return (w >> 16) & IDM; };
    auto tid_v = [](uint32_t w) { return w & IDM; };
    auto xmask = [](uint32_t w) { return ((w >> IDB) & 7u) | (((w >> (16 + IDB)) & 7u) << 3); };
    auto with_mask = [](uint32_t w, uint32_t m) { return w | ((m & 7u) << IDB) | ((m >> 3) << (16 + IDB)); };
    constexpr uint32_t SPARE = ~(IDM | (IDM << 16));
    auto nbr = [](uint32_t l, uint32_t d) -> uint32_t {
        const uint32_t a = d < 3 ? d : d - 3;
        const uint32_t step = 1u << (a == 0 ? 0 : a == 1 ? LX : LX + LY);
        return d < 3 ? l - step : l + step;
    };

    // 2. seed: T[l] = (l, first vertex of the closed in-tile neighbourhood)
    //    with l's lower neighbours in the spare bits; key histogram for the
    //    level buckets
    const uint32_t kmin_t = kmin, kmax_t = kmax;
    const float bscale = (float)BINS / ((float)(kmax_t - kmin_t) + 1.0f);
    auto bin_of = [&](uint32_t k) { return min((uint32_t)BINS - 1, (uint32_t)((float)(k - kmin_t) * bscale)); };
    for (uint32_t l = threadIdx.x; l < TV; l += NT) {
        if (!valid(l)) continue;
        const uint32_t lx = lxo(l), ly = lyo(l), lz = lzo(l);
        const uint32_t kl = K[l];
        uint32_t b = l, kb = kl;
        atomicAdd(&hist[bin_of(kb)], 1u);
        // candidates in ascending local index order: an earlier id wins ties,
        // so an earlier candidate replaces b only if strictly lower; a
        // neighbour is lower than l if its key is lower, or equal and its id
        // earlier (the -x, -y, -z neighbours)
        const uint32_t kmz = lz > 0 ? K[l - TX * TY] : 0xFFFFFFFFu, kmy = ly > 0 ? K[l - TX] : 0xFFFFFFFFu,
                       kmx = lx > 0 ? K[l - 1] : 0xFFFFFFFFu;
        const uint32_t kpx = lx + 1 < wx ? K[l + 1] : 0u, kpy = ly + 1 < wy ? K[l + TX] : 0u,
                       kpz = lz + 1 < wz ? K[l + TX * TY] : 0u;
        if (lz > 0 && kmz <= kb) b = l - TX * TY, kb = kmz;
        if (ly > 0 && kmy <= kb && (kmy < kb || l - TX < b)) b = l - TX, kb = kmy;
        if (lx > 0 && kmx <= kb && (kmx < kb || l - 1 < b)) b = l - 1, kb = kmx;
        if (lx + 1 < wx && kpx < kb) b = l + 1, kb = kpx;
        if (ly + 1 < wy && kpy < kb) b = l + TX, kb = kpy;
        if (lz + 1 < wz && kpz < kb) b = l + TX * TY, kb = kpz;
        const uint32_t lm = (uint32_t)(lx > 0 && kmx <= kl) | (uint32_t)(ly > 0 && kmy <= kl) << 1 |
                            (uint32_t)(lz > 0 && kmz <= kl) << 2 | (uint32_t)(lx + 1 < wx && kpx < kl) << 3 |
                            (uint32_t)(ly + 1 < wy && kpy < kl) << 4 | (uint32_t)(lz + 1 < wz && kpz < kl) << 5;
        T[l] = with_mask(sm_pack(l, b), lm);
    }
    __syncthreads();

    // 3. pointer jumping along the descent links (concurrent jumps only
    //    shorten chains, so racing readers stay correct); shortcuts start at
    //    the minima themselves. Bin -> bucket map from the histogram's
    //    prefix sums (monotone in the key).
    {
        volatile uint32_t *vT = T;
        for (uint32_t l = threadIdx.x; l < TV; l += NT) {
            if (!valid(l)) continue;
            const uint32_t w = vT[l];
            if (tid_v(w) == l) {
                SC[l] = (uint16_t)l;
                continue;
            }
            uint32_t x = tid_v(w);
            for (uint32_t h = 0; h < (uint32_t)TV; h++) {
                const uint32_t wx_ = vT[x];
                if (tid_v(wx_) == x) break;
                x = tid_v(wx_);
            }
            if (x != tid_v(w)) vT[l] = sm_pack(l, x) | (w & SPARE);
        }
        const uint32_t c = threadIdx.x < (uint32_t)BINS ? hist[threadIdx.x] : 0u;
        uint32_t incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        uint32_t before_w = 0;
        for (uint32_t w = 0; w < warp; w++) before_w += s_warp[w];
        if (threadIdx.x < (uint32_t)BINS)
            s_bmap[threadIdx.x] =
                (uint8_t)min((uint32_t)NB - 1, (uint32_t)(((uint64_t)(before_w + incl - c) * NB) / s_nvalid));
    }
    __syncthreads();
    volatile uint32_t *vT = T;
    auto bucket_of = [&](uint32_t k) { return (uint32_t)s_bmap[bin_of(k)]; };
    // The bucket of a key grows with the key, so "in bucket b or later" is
    // k >= s_thr[b], the smallest key of bucket b or after (kmax + 1 if none):
    // one compare in the shortcut climbs instead of the bin lookup. Read
    // only after the barriers that end step 4.
    if (threadIdx.x < (uint32_t)NB) {
        uint32_t lo = kmin_t, hi = kmax_t + 1u;
        while (lo < hi) {
            const uint32_t mid = lo + (hi - lo) / 2;
            if (bucket_of(mid) >= threadIdx.x) hi = mid;
            else lo = mid + 1;
        }
        s_thr[threadIdx.x] = lo;
    }
    // The cross masks of step 4 (from there on, until the bucket repair
    // rewrites the triplet) are kept in the same bits.

    // 4. cross masks, then a counting sort of the vertices by segment:
    //    inner vertices by level bucket (segments 0 .. NB-1), minima last
    //    (segment NB); the histogram is consumed, so the edge hash is cleared
    for (uint32_t i = threadIdx.x; i < (uint32_t)HS; i += NT) hkey[i] = 0xFFFFFFFFu, hlev[i] = ~0ull;
    for (uint32_t l = threadIdx.x; l < TV; l += NT) {
        if (!valid(l)) continue;
        const uint32_t w0 = vT[l];
        const uint32_t dl = tid_v(w0);
        if (dl == l) {  // a minimum
            atomicAdd(&s_bcur[NB], 1u);
            continue;
        }
        const uint32_t lm = xmask(w0);  // lower neighbours, from the seed
        uint32_t m = 0;
#pragma unroll
        for (uint32_t d = 0; d < 6; d++) {
            if (!((lm >> d) & 1u)) continue;
            const uint32_t w = nbr(l, d);
            if (tid_v(vT[w]) != dl) m |= 1u << d;  // w's minimum is another
        }
        atomicAdd(&s_bcur[bucket_of(K[l])], 1u);
        vT[l] = with_mask(sm_pack(l, dl), m);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int b = 0; b <= NB; b++) {
            s_boff[b] = run;
            run += s_bcur[b];
            s_bcur[b] = s_boff[b];
        }
        s_boff[NB + 1] = run;
    }
    __syncthreads();
    for (uint32_t l = threadIdx.x; l < TV; l += NT) {
        if (!valid(l)) continue;
        const uint32_t b = tid_v(vT[l]) == l ? (uint32_t)NB : bucket_of(K[l]);
        vlist[atomicAdd(&s_bcur[b], 1u)] = (uint16_t)l;  // order within a segment is free
    }
    __syncthreads();

    // 5. rounds over the level buckets
    bool ok = true;
    volatile uint16_t *vSC = SC;
    volatile uint32_t *vHK = hkey;
    volatile unsigned long long *vHL = hlev;
    // Round b's bucket repair (5c) runs in the same phase as round b+1's
    // scan (5a), with no barrier between them. The scan of round b stores in
    // every vertex of bucket b the round-b shortcut of its minimum, where its
    // repair starts, so the repair needs no shortcut cache; its climbs follow
    // links at or below the vertex's own level, which round b+1 never
    // changes (its merges, in the hash-crowded case run during the scan,
    // displace only links above bucket b). The scan reads the triplet of a
    // lower neighbour that the repair may be rewriting: before, (w, minimum)
    // or (w, shortcut); after, (w, representative) -- every one a vertex of
    // w's component below the round, with the same shortcut.
    for (int b = 0; b <= NB; b++) {
        // 5c. final tile triplets of the inner vertices of bucket b - 1 (this
        //     also clears their cross masks)
        if (b > 0) {
            for (uint32_t i = s_boff[b - 1] + threadIdx.x; i < s_boff[b]; i += NT) {
                const uint32_t l = vlist[i];
                uint32_t wr;
                const uint32_t r = sm_climb<TV>(T, K, tid_v(vT[l]), l, K[l], wr, ok);
                T[l] = sm_pack(l, r);
            }
        }
        if (b == NB) {
            // 6. repair the branch minima (Algorithm 5), beside the last
            //    bucket repair: both only follow links of minima, and a
            //    minimum's repair moves its target along its own chain below
            //    its own saddle, which leaves every climb's result unchanged
            for (uint32_t i = s_boff[NB] + threadIdx.x; i < s_boff[NB + 1]; i += NT) {
                const uint32_t l = vlist[i];
                const uint32_t w = vT[l];
                const uint32_t s = sm_s(w);
                if (s == l) continue;  // inner vertex or root
                uint32_t wr;
                const uint32_t r = sm_climb<TV>(T, K, sm_v(w), s, K[s], wr, ok);
                if (r != sm_v(w)) T[l] = sm_pack(s, r);
            }
            break;
        }
        // shortcut of minimum m for round b: climb through the links whose
        // saddle lies in an earlier bucket, from where round (SC >> IDB) left it
        auto shortcut = [&](uint32_t m) -> uint32_t {
            const uint32_t sc = vSC[m];
            uint32_t x = sc & IDM;
            if ((sc >> IDB) == (uint32_t)b) return x;
            for (uint32_t h = 0; h < (uint32_t)TV; h++) {
                const uint32_t w = vT[x];
                if (w == sm_pack(x, x) || K[sm_s(w)] >= s_thr[b]) break;
                x = sm_v(w);
            }
            vSC[m] = (uint16_t)(((uint32_t)b << IDB) | x);
            return x;
        };
        // 5a. scan the cross edges whose upper end S lies in bucket b; collect
        //     those whose ends are not yet known to be connected below S,
        //     one per pair of shortcuts (the earliest S); store every
        //     vertex's shortcut for its repair
        for (uint32_t i = s_boff[b] + threadIdx.x; i < s_boff[b + 1]; i += NT) {
            const uint32_t S = vlist[i];
            const uint32_t TSw = vT[S];
            uint32_t m = xmask(TSw);
            const uint32_t aS = shortcut(tid_v(TSw));
            vT[S] = sm_pack(S, aS);
            if (m == 0) continue;
            const uint32_t kS = K[S];
            do {
                const uint32_t d = __ffs(m) - 1;
                m &= m - 1;
                const uint32_t w = nbr(S, d);
                const uint32_t Tw = vT[w];
                // a vertex of w's component below the round: an inner
                // vertex's target, else w itself
                const uint32_t dw = (tid_s(Tw) == w && tid_v(Tw) != w) ? tid_v(Tw) : w;
                const uint32_t aw = shortcut(dw);
                if (aw == aS) continue;  // already connected below S
                const uint32_t pr = aS < aw ? (aS << IDB) | aw : (aw << IDB) | aS;
                const unsigned long long lev = ((unsigned long long)kS << 32) | S;
                uint32_t h = (pr * 0x9E3779B1u) >> (32 - HLOG);
                bool placed = false;
                for (uint32_t p = 0; p < kTileHashProbes; p++) {
                    uint32_t k0 = vHK[h];
                    if (k0 == 0xFFFFFFFFu) k0 = atomicCAS(hkey + h, 0xFFFFFFFFu, pr);
                    if (k0 == 0xFFFFFFFFu || k0 == pr) {  // the pair's slot: keep the earliest level
                        if (vHL[h] > lev) atomicMin(hlev + h, lev);
                        placed = true;
                        break;
                    }
                    h = (h + 1) & (HS - 1);
                }
                if (!placed) sm_merge<TV>(T, K, S, kS, aS, aw, ok);  // hash crowded: merge in place
            } while (m);
        }
        __syncthreads();
        // 5b. run the collected merges side by side and clear the hash
        for (uint32_t i = threadIdx.x; i < (uint32_t)HS; i += NT) {
            const uint32_t pr = hkey[i];
            if (pr == 0xFFFFFFFFu) continue;
            const unsigned long long lev = hlev[i];
            hkey[i] = 0xFFFFFFFFu, hlev[i] = ~0ull;
            sm_merge<TV>(T, K, (uint32_t)lev, (uint32_t)(lev >> 32), pr >> IDB, pr & IDM, ok);
        }
        __syncthreads();
    }
    if (!ok) raise_status(status, ST_TIMEOUT);
    __syncthreads();

    // 6b. for k_cross: the tile-local top of every face vertex at the level
    //     of its edge into the neighbouring tile, i.e. the deepest vertex of
    //     its tile component below that level. Levels compare (key, global
    //     id), since the other end lies outside the tile. Face buffer of a
    //     tile: +x, +y, +z, then -x, -y, -z faces, each indexed by the two
    //     in-face coordinates on the full tile extent.
    if (!WIDE && fd.faces) {
        constexpr uint32_t FX = TY * TZ, FY = TX * TZ, FZ = TX * TY, FH = FX + FY + FZ;
        uint32_t *out = fd.faces + (size_t)tile * (2 * FH);
        const uint32_t has_n = (uint32_t)(x0 + TX < nx) | (uint32_t)(y0 + TY < ny) << 1 |
                               (uint32_t)(z0 + TZ < nz) << 2 | (uint32_t)(x0 > 0) << 3 | (uint32_t)(y0 > 0) << 4 |
                               (uint32_t)(z0 > 0) << 5;
        for (uint32_t e = threadIdx.x; e < 2 * FH; e += NT) {
            const uint32_t side = e / FH, r = e - side * FH;  // side 0: + faces, 1: - faces
            uint32_t dir, lx, ly, lz;
            if (r < FX) dir = 0, ly = r % TY, lz = r / TY, lx = side ? 0 : TX - 1;
            else if (r < FX + FY) dir = 1, lx = (r - FX) % TX, lz = (r - FX) / TX, ly = side ? 0 : TY - 1;
            else dir = 2, lx = (r - FX - FY) % TX, ly = (r - FX - FY) / TX, lz = side ? 0 : TZ - 1;
            if (!((has_n >> (dir + 3 * side)) & 1u) || lx >= wx || ly >= wy || lz >= wz) continue;
            const uint32_t l = lx + TX * (ly + TY * lz);
            const uint32_t ga = gid(l);
            const uint32_t step = dir == 0 ? 1u : dir == 1 ? nx : nxy;
            const uint32_t gb = side ? ga - step : ga + step;
            const uint32_t kb = order_key(sg * __ldg(f + gb)), ka = K[l];
            uint32_t kS = ka, gS = ga;  // level: the later end of the edge
            if (kbefore(ka, ga, kb, gb)) kS = kb, gS = gb;
            uint32_t x = l;
            for (uint32_t h = 0; h < (uint32_t)TV; h++) {
                const uint32_t w = vT[x];
                if (w == sm_pack(x, x)) break;
                const uint32_t sv = sm_s(w);
                if (kbefore(kS, gS, K[sv], gid(sv))) break;  // link above the level
                x = sm_v(w);
            }
            out[e] = gid(x);
        }
    }

    // 7. write the tile's triplets with global ids (coalesced rows)
    if constexpr (WIDE) {
        for (uint32_t l = threadIdx.x; l < TV; l += NT) {
            if (!valid(l)) continue;
            const uint32_t w = T[l];
            reinterpret_cast<ulonglong2 *>(W)[gid(l)] = make_ulonglong2(gid(sm_s(w)), gid(sm_v(w)));
        }
    } else if (vec) {
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

// One CTA per tile (queue == null), or a persistent grid that takes tiles
// from a device-side counter until none is left (the batched build). FULL is
// set when every tile lies inside the grid (grid sides multiples of the tile
// sides), which drops all partial-tile bounds checks.
template <int LX, int LY, int LZ, int NT, int NB, class Loc, bool FULL, bool WIDE = false>
__global__ void __launch_bounds__(NT, NT >= 1024 ? 2 : NT == 512 ? 4 : 1536 / NT) k_tile(Loc loc, uint32_t ntiles, uint32_t *queue,
                                                                      uint32_t *status)
{
    if (queue == nullptr) {
        uint32_t local;
        const FieldDesc fd = loc.tile(blockIdx.x, local);
        tile_body<LX, LY, LZ, NT, NB, FULL, WIDE>(fd, local, status);
        return;
    }
    __shared__ uint32_t s_next;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(queue, 1u);
        __syncthreads();
        const uint32_t t = s_next;
        __syncthreads();
        if (t >= ntiles) break;
        uint32_t local;
        const FieldDesc fd = loc.tile(t, local);
        tile_body<LX, LY, LZ, NT, NB, FULL>(fd, local, status);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- k_cross
//
// The rest of the edge loop of Algorithm 1: the edges between neighbouring
// tiles, merged with 64-bit CAS on the global triplets (Algorithms 2, 3).
// CTA t takes the edges from tile t to its +x, +y, +z neighbour tiles. k_tile
// left, for both ends of every such edge (a, b) at level S, the tile-local
// top of the end at S (the deepest vertex of its tile component below S). Two
// edges whose ends have the same pair of tops join the same two tile
// components, and the later of the two is already represented once the
// earlier is merged, so the CTA keeps, per pair of tops, only the edge with
// the earliest level (a shared-memory hash with 64-bit atomicMin on
// (key, id) of S) and merges that one, starting its climbs at the tops.
//
// Pairs from different faces never coincide (their second tops lie in
// different neighbour tiles), so the three faces go through one small hash
// in turn: fill it with the face's edges, then each edge that still holds
// its slot's minimum (S identifies an edge within a face) lists itself and
// clears the slot. The merges then run from the list, one per thread, all
// lanes busy; the small footprint lets 8 CTAs share an SM.
constexpr uint32_t kCrossHash = 1024;

template <int LX, int LY, int LZ, class Loc>
__global__ void __launch_bounds__(256, 8) k_cross(Loc loc, uint32_t *status)
{
    if (block_skips(status)) return;
    using TS = Tile<LX, LY, LZ>;
    constexpr uint32_t TX = TS::TX, TY = TS::TY, TZ = TS::TZ;
    constexpr uint32_t FX = TY * TZ, FY = TX * TZ, FZ = TX * TY, FH = FX + FY + FZ;
    constexpr uint32_t FMAX = FX > FY ? (FX > FZ ? FX : FZ) : (FY > FZ ? FY : FZ);
    constexpr uint32_t PER = (FMAX + 255) / 256;  // edges of one face per thread
    static_assert(FMAX <= kCrossHash / 3 * 2, "hash load factor");
    static_assert(FH <= 65536, "16-bit face edge indices");
    constexpr unsigned long long EMPTY = ~0ull;
    __shared__ unsigned long long hkey[kCrossHash], hval[kCrossHash];
    __shared__ uint32_t todo_s[FH];  // the saddle S of each edge to merge
    __shared__ uint16_t todo_e[FH];  // and its face edge index
    __shared__ uint32_t s_ntodo;
    uint32_t tile;
    const FieldDesc fd = loc.tile(blockIdx.x, tile);
    uint64_t *W = fd.W;
    const Field f{fd.f, fd.sg};
    const uint32_t nx = fd.nx, ny = fd.ny, nz = fd.nz, ntx = fd.ntx, nty = fd.nty;
    const uint32_t tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
    const uint32_t x0 = tx * TX, y0 = ty * TY, z0 = tz * TZ;
    const uint32_t wx = min(TX, nx - x0), wy = min(TY, ny - y0), wz = min(TZ, nz - z0);
    const uint32_t nxy = nx * ny;
    const uint32_t base = z0 * nxy + y0 * nx + x0;
    const uint32_t *fa = fd.faces + (size_t)tile * (2 * FH);
    const uint32_t *fbx = fd.faces + (size_t)(tile + 1) * (2 * FH) + FH;
    const uint32_t *fby = fd.faces + (size_t)(tile + ntx) * (2 * FH) + FH + FX;
    const uint32_t *fbz = fd.faces + (size_t)(tile + ntx * nty) * (2 * FH) + FH + FX + FY;
    const bool hx = x0 + TX < nx, hy = y0 + TY < ny, hz = z0 + TZ < nz;
    // edge e of the +x, +y, +z faces: its ends (a in this tile, b in the
    // neighbour) and their tops; false where the edge does not exist
    auto edge = [&](uint32_t e, uint32_t &a, uint32_t &b, uint32_t &ta, uint32_t &tb) -> bool {
        if (e < FX) {
            const uint32_t ly = e % TY, lz = e / TY;
            if (!hx || ly >= wy || lz >= wz) return false;
            a = base + lz * nxy + ly * nx + (TX - 1);
            b = a + 1;
            tb = fbx[e];
        } else if (e < FX + FY) {
            const uint32_t k = e - FX, lx = k % TX, lz = k / TX;
            if (!hy || lx >= wx || lz >= wz) return false;
            a = base + lz * nxy + (TY - 1) * nx + lx;
            b = a + nx;
            tb = fby[k];
        } else {
            const uint32_t k = e - FX - FY, lx = k % TX, ly = k / TX;
            if (!hz || lx >= wx || ly >= wy) return false;
            a = base + (TZ - 1) * nxy + ly * nx + lx;
            b = a + nxy;
            tb = fbz[k];
        }
        ta = fa[e];
        return true;
    };
    for (uint32_t i = threadIdx.x; i < kCrossHash; i += blockDim.x) hkey[i] = EMPTY, hval[i] = EMPTY;
    if (threadIdx.x == 0) s_ntodo = 0;
    __syncthreads();
    for (uint32_t face = 0; face < 3; face++) {
        const uint32_t e0 = face == 0 ? 0 : face == 1 ? FX : FX + FY;
        const uint32_t e1 = face == 0 ? FX : face == 1 ? FX + FY : FH;
        uint32_t slot[PER];
        unsigned long long mine[PER];
#pragma unroll
        for (uint32_t q = 0; q < PER; q++) {
            const uint32_t e = e0 + q * 256 + threadIdx.x;
            mine[q] = EMPTY;
            uint32_t a, b, ta, tb;
            if (e >= e1 || !edge(e, a, b, ta, tb)) continue;
            const float va = f[a], vb = f[b];
            const uint32_t S = before(vb, b, va, a) ? a : b;
            const float vS = S == a ? va : vb;
            const unsigned long long key = ((unsigned long long)ta << 32) | tb;
            const uint32_t bits = vS == 0.0f ? 0u : __float_as_uint(vS);
            const uint32_t kS = (bits & 0x80000000u) ? ~bits : (bits | 0x80000000u);
            mine[q] = ((unsigned long long)kS << 32) | S;
            uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 54) & (kCrossHash - 1);
            for (uint32_t p = 0; p < kCrossHash; p++) {
                const unsigned long long k0 = atomicCAS(&hkey[h], EMPTY, key);
                if (k0 == EMPTY || k0 == key) {
                    atomicMin(&hval[h], mine[q]);
                    break;
                }
                h = (h + 1) & (kCrossHash - 1);
            }
            slot[q] = h;
        }
        __syncthreads();
        // the winner of each slot lists its edge and clears the slot
#pragma unroll
        for (uint32_t q = 0; q < PER; q++) {
            if (mine[q] == EMPTY || hval[slot[q]] != mine[q]) continue;
            const uint32_t j = atomicAdd(&s_ntodo, 1u);
            todo_s[j] = (uint32_t)mine[q];
            todo_e[j] = (uint16_t)(e0 + q * 256 + threadIdx.x);
            hkey[slot[q]] = EMPTY, hval[slot[q]] = EMPTY;
        }
        __syncthreads();
    }
    bool ok = true;
    for (uint32_t j = threadIdx.x; j < s_ntodo; j += blockDim.x) {
        uint32_t a, b, ta, tb;
        edge(todo_e[j], a, b, ta, tb);
        ok &= merge(W, f, todo_s[j], ta, tb);
    }
    if (!ok) raise_status(status, ST_TIMEOUT);
}

// --------------------------------------------------------------- k_repair
//
// Repair (Algorithm 5) after the cross-tile merges: T[u] = (s, Rep(u, s))
// restores minimality. Level comparisons use the vertex order, not values
// alone: with tied values a saddle s' equal in value to s but after it in the
// order is not yet part of the sublevel set at s. Concurrent repairs only
// replace a target by one further along the same chain below the same level,
// so a stale copy of an entry is still a valid (longer) way to the same
// answer: every chase here uses ordinary cached loads.
//
// One CTA per tile, in four steps:
//  1. scan the tile: collect its branch minima (s != u) in a list, and enter
//     the target v of every inner vertex (s == u != v) in a shared-memory
//     hash of targets (about 360 distinct targets serve the 7,400 inner
//     vertices of a tile on the 1024^3 lognormal field);
//  2. give each hashed target a slot for a copy of its chain;
//  3. repair the branch minima, and copy the first kHops links of the chain
//     of every hashed target into its slot, with the order keys of their
//     saddles (one loop over both kinds of work, all lanes busy). A link
//     whose saddle is not above the one before is folded into it (whoever
//     passed the earlier saddle passes this one too), so the saddles of a
//     copy increase strictly;
//  4. repair every inner vertex: a binary search in its target's copy finds
//     the last link at or below it, and only when the whole copy lies below
//     it does the walk go on along the global chain.
// Steps 1 and 4 load four rows per thread before using any, so that the
// loads of a thread overlap. A branch minimum that finds the list full is
// marked in a bitmap in step 1 and repaired in step 3 (kept out of the
// unrolled row loop); a target without a slot (hash or copies full) is
// chased along the global chain in step 4.
//
// With LAB the pass also labels the components of G_t (the labels of
// k_labels) where it already stands. The representative of u at level t is
// the end of the walk from u along links with f(s) <= t (Algorithm 4 with a
// value test). Any valid triplet forest gives the same end, repaired or not:
// a walk stops at the first link above t, and every link it passes joins two
// vertices of one component of G_t, the second deeper. So a branch minimum
// continues the walk from its repaired target when its saddle is at or below
// t (step 3), every copied chain gives its target's label by a search of the
// copy for t, shared by all inner vertices of the target (step 3), and step 4
// writes every vertex's label: 0xFFFFFFFF above t, the copy's label, or a
// global walk for a target without a copy. Concurrent repairs move entries
// along their own chains below their own saddles, which keeps every walk's
// end.
// The label at t of the component reached from x: the end r of the walk
// along links with f(s) <= t (Algorithm 4 with a value test), or 0xFFFFFFFF
// when eps > 0 and r heads a branch of persistence below eps (its component
// lies in a filled pit). Bit 32 of the result is set if the walk ran out of
// steps. Out of line: the callers take it for a minority of vertices, and
// inlined copies in their unrolled loops slow the common path.
__device__ __noinline__ uint64_t label_walk(const uint64_t *W, const Field f, uint32_t x, float t, float eps)
{
    for (uint32_t h = 0;; h++) {
        const uint64_t T = W[x];
        const uint32_t s = tri_s(T), v = tri_v(T);
        if ((s == x && v == x) || !(f[s] <= t)) break;
        x = v;
        if (h >= kChaseLimit) return (1ull << 32) | x;
    }
    if (eps > 0.0f) {
        const uint32_t s = tri_s(W[x]);
        if (s != x && !(f[s] - f[x] >= eps)) return 0xFFFFFFFFull;
    }
    return x;
}

// Representative(x, u) for an inner vertex whose target's copy does not reach
// its level (Algorithm 4 along the global chain); bit 32 set if the walk ran
// out of steps. Out of line for the same reason as label_walk.
__device__ __noinline__ uint64_t repair_walk(const uint64_t *W, const Field f, uint32_t x, uint32_t u, float fu)
{
    uint32_t steps = 0;
    const uint32_t r = representative_cached(W, f, x, u, fu, steps);
    return steps > kChaseLimit ? (1ull << 32) | r : r;
}

template <int LX, int LY, int LZ>
struct RepairShape {
    static constexpr uint32_t TV = 1u << (LX + LY + LZ);
    static constexpr uint32_t kHops = 8;          // links copied per target
    static constexpr uint32_t kCap = TV / 16 / kRepairShrink;   // copies
    static constexpr uint32_t kHash = TV / 8 / kRepairShrink;   // hash slots for targets
    static constexpr uint32_t kList = TV / 4 / kRepairShrink;   // branch minima listed
    static constexpr size_t kSmem = (size_t)kCap * kHops * 12 + (size_t)kHash * 4 + (size_t)kHash * 2 +
                                    (size_t)kList * 2 + (size_t)kCap * 2 + (size_t)TV / 8;
    static constexpr size_t kSmemLab = kSmem + (size_t)kCap * 4;  // + each copy's label
};

template <int LX, int LY, int LZ, int NT, class Loc, bool LAB>
__global__ void __launch_bounds__(NT, 3) k_repair(Loc loc, uint32_t *status, const LabelArgs la)
{
    if (block_skips(status)) return;
    using RS = RepairShape<LX, LY, LZ>;
    constexpr uint32_t TX = 1u << LX, TY = 1u << LY, TV = RS::TV, H = RS::kHops, CAP = RS::kCap,
                       HS = RS::kHash, LIST = RS::kList;
    constexpr uint32_t NB = 4;  // rows loaded together
    static_assert(TV % (NT * NB) == 0, "whole batches of rows");
    static_assert((H & (H - 1)) == 0 && (HS & (HS - 1)) == 0, "powers of two");
    static_assert((HS + LIST + CAP) % 2 == 0, "the bitmap after the 16-bit arrays is 4-byte aligned");
    constexpr uint32_t EMPTY = 0xFFFFFFFFu;  // free hash slot (not a vertex id: ids are < n < 2^32 - 1)
    constexpr uint32_t END = 0xFFFFFFFFu;    // copied saddle after the chain's root: above every (key, id)
    constexpr uint16_t NOSLOT = 0xFFFFu;
    constexpr uint32_t kProbes = 16;
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *es = smem;                       // copied links: saddle, its key, target
    uint32_t *ek = es + CAP * H;
    uint32_t *ev = ek + CAP * H;
    uint32_t *hkey = ev + CAP * H;             // hashed targets
    uint32_t *slab = hkey + HS;                // LAB: label at t of each copy's target
    uint16_t *hslot = reinterpret_cast<uint16_t *>(slab + (LAB ? CAP : 0));  // copy slots of the targets
    uint16_t *list = hslot + HS;               // branch minima (tile-local ids)
    uint16_t *cslot = list + LIST;             // hash slot of each copy's target
    uint32_t *ovf = reinterpret_cast<uint32_t *>(cslot + CAP);  // bit per vertex: minima past the list
    __shared__ uint32_t s_nmin, s_ncopy;

    uint32_t tile;
    const FieldDesc fd = loc.tile(blockIdx.x, tile);
    uint64_t *W = fd.W;
    const Field f{fd.f, fd.sg};
    const uint32_t nx = fd.nx, ny = fd.ny, nz = fd.nz, ntx = fd.ntx, nty = fd.nty;
    const uint32_t tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
    const uint32_t x0 = tx * TX, y0 = ty * TY, z0 = tz * (1u << LZ);
    const uint32_t wx = min(TX, nx - x0), wy = min(TY, ny - y0), wz = min(1u << LZ, nz - z0);
    const uint32_t nxy = nx * ny;
    const uint32_t base = z0 * nxy + y0 * nx + x0;
    const uint32_t lane = threadIdx.x & 31;
    auto gid_of = [&](uint32_t l) {
        return base + (l >> (LX + LY)) * nxy + ((l >> LX) & (TY - 1)) * nx + (l & (TX - 1));
    };
    auto inside = [&](uint32_t l) {
        return (l & (TX - 1)) < wx && ((l >> LX) & (TY - 1)) < wy && (l >> (LX + LY)) < wz;
    };
    auto hash0 = [](uint32_t v) { return (v * 0x9E3779B1u) >> (32 - log2i(HS)); };
    // slot of target v in the hash, HS if absent
    auto find = [&](uint32_t v) -> uint32_t {
        uint32_t h = hash0(v);
        for (uint32_t p = 0; p < kProbes; p++) {
            const uint32_t k = hkey[h];
            if (k == v) return h;
            if (k == EMPTY) return HS;
            h = (h + 1) & (HS - 1);
        }
        return HS;
    };

    bool ok = true;
    constexpr uint32_t OUT = 0xFFFFFFFFu;  // label of a vertex outside G_t (or in a filled pit)
    const float lt = la.t;
    // label at t reached from x: x itself when x is known to head its
    // component (walk false) and eps <= 0, else label_walk
    auto label_from = [&](uint32_t x, bool walk) -> uint32_t {
        if (!walk && !(la.eps > 0.0f)) return x;
        const uint64_t r = label_walk(W, f, x, lt, la.eps);
        if (r >> 32) ok = false;
        return (uint32_t)r;
    };
    // label of branch minimum m (saddle value fs) whose link leads to r
    auto min_label = [&](uint32_t m, float fs, uint32_t r) { return fs <= lt ? label_from(r, true) : label_from(m, false); };

    for (uint32_t i = threadIdx.x; i < HS; i += NT) hkey[i] = EMPTY;
    for (uint32_t i = threadIdx.x; i < TV / 32; i += NT) ovf[i] = 0;
    if (threadIdx.x == 0) s_nmin = 0, s_ncopy = 0;
    __syncthreads();

    // 1. scan
    volatile uint32_t *vhk = hkey;
    for (uint32_t l0 = 0; l0 < TV; l0 += NT * NB) {
        uint64_t Tb[NB];
#pragma unroll
        for (uint32_t k = 0; k < NB; k++) {
            const uint32_t l = l0 + k * NT + threadIdx.x;
            const uint32_t u = gid_of(l);
            Tb[k] = inside(l) ? W[u] : tri_pack(u, u);
        }
#pragma unroll
        for (uint32_t k = 0; k < NB; k++) {
            const uint32_t l = l0 + k * NT + threadIdx.x;
            const uint32_t u = gid_of(l);
            const uint32_t s = tri_s(Tb[k]), v = tri_v(Tb[k]);
            const bool is_min = s != u;
            if (!is_min && v != u) {  // inner vertex: hash its target
                uint32_t h = hash0(v);
                for (uint32_t p = 0; p < kProbes; p++) {
                    uint32_t kk = vhk[h];
                    if (kk == EMPTY) kk = atomicCAS(hkey + h, EMPTY, v);
                    if (kk == EMPTY || kk == v) break;
                    h = (h + 1) & (HS - 1);
                }
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, is_min);
            if (bal) {
                uint32_t pos = 0;
                if (lane == 0) pos = atomicAdd(&s_nmin, __popc(bal));
                pos = __shfl_sync(0xffffffffu, pos, 0) + __popc(bal & ((1u << lane) - 1u));
                if (is_min && pos < LIST) {
                    list[pos] = (uint16_t)l;
                } else if (is_min) {  // list full: mark it for step 3
                    atomicOr(&ovf[l >> 5], 1u << (l & 31));
                }
            }
        }
    }
    __syncthreads();

    // 2. copy slots for the hashed targets
    for (uint32_t i = threadIdx.x; i < HS; i += NT) {
        if (hkey[i] == EMPTY) continue;
        const uint32_t c = atomicAdd(&s_ncopy, 1u);
        hslot[i] = c < CAP ? (uint16_t)c : NOSLOT;
        if (c < CAP) cslot[c] = (uint16_t)i;
    }
    __syncthreads();

    // 3. branch minima (items below nmin) and copies of target chains (one
    //    item per copy: copy c serves the target in hash slot cslot[c])
    // Repair of the branch minimum with local id l (and with LAB its label,
    // which step 4 overwrites with 0xFFFFFFFF above t)
    auto repair_min = [&](uint32_t l) {
        const uint32_t u = gid_of(l);
        const uint64_t T = W[u];
        const uint32_t s = tri_s(T), t = tri_v(T);
        uint32_t steps = 0;
        const float fs = f[s];
        const uint32_t r = representative_cached(W, f, t, s, fs, steps);
        if (steps > kChaseLimit) ok = false;
        else if (r != t) st_tri(W + u, tri_pack(s, r));
        if (LAB) la.labels[u] = min_label(u, fs, r);
    };
    // items: the listed minima, the copies, then (when the list overflowed)
    // the words of the bitmap of the minima past it; the two kinds of minima
    // share one call of repair_min, so that its code appears once
    const uint32_t nmin = min(s_nmin, LIST), ncopy = min(s_ncopy, CAP);
    const uint32_t nover = s_nmin > LIST ? TV / 32 : 0;
    for (uint32_t i = threadIdx.x; i < nmin + ncopy + nover; i += NT) {
        if (i < nmin || i >= nmin + ncopy) {
            const bool listed = i < nmin;
            const uint32_t w = i - nmin - ncopy;
            for (uint32_t m = listed ? 1u : ovf[w]; m; m &= m - 1)
                repair_min(listed ? (uint32_t)list[i] : w * 32 + __ffs(m) - 1);
            continue;
        }
        const uint32_t c = i - nmin;  // copy c, of the target in hash slot cslot[c]
        const uint32_t x0v = hkey[cslot[c]];
        const uint32_t b = c * H;
        uint32_t x = x0v, j = 0;
        bool ended = false;
        uint64_t T = W[x];
        for (uint32_t step = 0; step < 4 * H && j < H; step++) {
            const uint32_t s = tri_s(T), v = tri_v(T);
            if (s == x && v == x) {  // a root: the chain ends
                ended = true;
                break;
            }
            const float fs = f[s];
            const uint64_t Tn = W[v];  // loaded together with the saddle's value
            const uint32_t ks = order_key(fs);
            if (j > 0 && !kbefore(ek[b + j - 1], es[b + j - 1], ks, s)) {
                ev[b + j - 1] = v;  // not above the previous saddle: fold
            } else {
                es[b + j] = s, ek[b + j] = ks, ev[b + j] = v;
                j++;
            }
            x = v;
            T = Tn;
        }
        // pad: after a root with END (above every level); when the copy
        // stops short of the root, with the last link again, leading to x
        // where a vertex above it goes on along the global chain
        const uint32_t ps = ended ? END : es[b + j - 1], pk = ended ? END : ek[b + j - 1];
        for (; j < H; j++) es[b + j] = ps, ek[b + j] = pk, ev[b + j] = x;
        if (LAB) {
            // links of the copy at or below t (saddle values; END is above
            // every finite key); past the whole copy the walk goes on globally
            const uint32_t kt = order_key(lt);
            uint32_t lo = 0;
            while (lo < H && ek[b + lo] <= kt) lo++;
            slab[c] = label_from(lo ? ev[b + lo - 1] : x0v, lo == H);
        }
    }
    __syncthreads();

    // 4. inner vertices
    for (uint32_t l0 = 0; l0 < TV; l0 += NT * NB) {
        uint64_t Tb[NB];
        float fb[NB];
#pragma unroll
        for (uint32_t k = 0; k < NB; k++) {
            const uint32_t l = l0 + k * NT + threadIdx.x;
            const uint32_t u = gid_of(l);
            const bool in = inside(l);
            Tb[k] = in ? W[u] : tri_pack(u, u);
            fb[k] = in ? f[u] : 0.0f;
        }
#pragma unroll
        for (uint32_t k = 0; k < NB; k++) {
            const uint32_t l = l0 + k * NT + threadIdx.x;
            const uint32_t u = gid_of(l);
            const uint32_t s = tri_s(Tb[k]), t = tri_v(Tb[k]);
            if (s != u || t == u) {  // a branch minimum, the root, or outside the grid
                if (LAB && inside(l)) {
                    if (!(fb[k] <= lt)) la.labels[u] = OUT;
                    else if (s == u) la.labels[u] = u;  // the root labels itself
                }
                continue;
            }
            const uint32_t h = find(t);
            const uint16_t c = h < HS ? hslot[h] : NOSLOT;
            uint32_t r = t;
            bool global = true;
            if (c != NOSLOT) {
                const uint32_t b = (uint32_t)c * H;
                const uint32_t ku = order_key(fb[k]);
                // number of copied links at or below u (saddles increase)
                uint32_t lo = 0;
#pragma unroll
                for (uint32_t w = H / 2; w > 0; w >>= 1)
                    if (!kbefore(ku, u, ek[b + lo + w - 1], es[b + lo + w - 1])) lo += w;
                if (lo < H && !kbefore(ku, u, ek[b + lo], es[b + lo])) lo++;
                if (lo > 0) r = ev[b + lo - 1];
                global = lo == H;
            }
            if (global) {
                const uint64_t rr = repair_walk(W, f, r, u, fb[k]);
                if (rr >> 32) {
                    ok = false;
                    continue;
                }
                r = (uint32_t)rr;
            }
            if (r != t) st_tri(W + u, tri_pack(u, r));
            // t >= f(u): the walk at t passes the representative at u
            if (LAB) la.labels[u] = !(fb[k] <= lt) ? OUT : c != NOSLOT ? slab[c] : label_from(r, true);
        }
    }
    if (!ok) raise_status(status, ST_TIMEOUT);
}

// ------------------------------------------------------------ host side

// Tile shapes. Variant 0: 16 x 16 x 16, 4096 vertices, about 53 KiB of
// shared memory, four CTAs of 512 threads per SM (32 x 16 x 16 tiles in two
// CTAs of 1024 threads run the tile kernel 6 % slower on the 1024^3 field:
// with four CTAs per SM, one CTA's round barrier leaves three others to
// issue). Variant 1: 16 x 16 x 8, 2048 vertices, about 26 KiB, six CTAs of
// 256 threads per SM, for batches of small fields that would leave most of a
// large tile empty. 8 level buckets in both. Variant 2: 32 x 16 x 16 bricks
// of 8192 vertices, the unit of the repair pass of a single field (its
// shared-memory copies of target chains serve twice as many vertices as in
// a 16^3 brick) and of the wide-id tile kernel.
constexpr int kBuckets = 8;
template <int V> struct Variant;
template <> struct Variant<0> { static constexpr int LX = 4, LY = 4, LZ = 4, NT = 512; };
template <> struct Variant<1> { static constexpr int LX = 4, LY = 4, LZ = 3, NT = 256; };
template <> struct Variant<2> { static constexpr int LX = 5, LY = 4, LZ = 4, NT = 1024; };

void tile_shape(int variant, uint32_t &tx, uint32_t &ty, uint32_t &tz)
{
    if (variant == 1) {
        tx = 1u << Variant<1>::LX, ty = 1u << Variant<1>::LY, tz = 1u << Variant<1>::LZ;
    } else if (variant == 2) {
        tx = 1u << Variant<2>::LX, ty = 1u << Variant<2>::LY, tz = 1u << Variant<2>::LZ;
    } else {
        tx = 1u << Variant<0>::LX, ty = 1u << Variant<0>::LY, tz = 1u << Variant<0>::LZ;
    }
}

uint32_t face_words(int variant)
{
    uint32_t tx, ty, tz;
    tile_shape(variant, tx, ty, tz);
    return 2 * (ty * tz + tx * tz + tx * ty);
}

uint64_t tile_count(int variant, uint32_t nx, uint32_t ny, uint32_t nz)
{
    uint32_t tx, ty, tz;
    tile_shape(variant, tx, ty, tz);
    return (uint64_t)((nx + tx - 1) / tx) * ((ny + ty - 1) / ty) * ((nz + tz - 1) / tz);
}

template <int V, int NB, class Loc, bool FULL>
static cudaError_t tile_attrs()
{
    using VV = Variant<V>;
    using TS = Tile<VV::LX, VV::LY, VV::LZ, VV::NT>;
    static AttrFlags flags;  // per instantiation
    int dev;
    if (!flags.pending(dev)) return cudaSuccess;
    auto ktile = k_tile<VV::LX, VV::LY, VV::LZ, VV::NT, NB, Loc, FULL>;
    cudaError_t e = cudaFuncSetAttribute(ktile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TS::kSmem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(ktile, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    flags.done(dev);
    return cudaSuccess;
}

template <int V, int NT, class Loc, bool LAB>
static cudaError_t repair_attrs()
{
    using VV = Variant<V>;
    using RS = RepairShape<VV::LX, VV::LY, VV::LZ>;
    static AttrFlags flags;  // per instantiation
    int dev;
    if (!flags.pending(dev)) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(k_repair<VV::LX, VV::LY, VV::LZ, NT, Loc, LAB>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(LAB ? RS::kSmemLab : RS::kSmem));
    if (e == cudaSuccess) flags.done(dev);
    return e;
}

// The tile kernel with NB level buckets (merge rounds); FULL only for a
// single field whose sides are multiples of the tile's.
template <int V, int NB, class Loc>
static cudaError_t launch_tile(const Loc &loc, uint32_t ntiles, uint32_t *queue, int persistent_grid, bool full,
                               uint32_t *status, cudaStream_t st)
{
    using VV = Variant<V>;
    using TS = Tile<VV::LX, VV::LY, VV::LZ, VV::NT>;
    const unsigned grid = queue ? (unsigned)persistent_grid : ntiles;
    cudaError_t e;
    if constexpr (std::is_same<Loc, OneField>::value) {  // batches never take the FULL form
        if (full) {
            if ((e = tile_attrs<V, NB, Loc, true>()) != cudaSuccess) return e;
            k_tile<VV::LX, VV::LY, VV::LZ, VV::NT, NB, Loc, true><<<grid, VV::NT, TS::kSmem, st>>>(loc, ntiles,
                                                                                               queue, status);
            count_launch();
            return cudaGetLastError();
        }
    }
    {
        if ((e = tile_attrs<V, NB, Loc, false>()) != cudaSuccess) return e;
        k_tile<VV::LX, VV::LY, VV::LZ, VV::NT, NB, Loc, false><<<grid, VV::NT, TS::kSmem, st>>>(loc, ntiles, queue,
                                                                                            status);
    }
    count_launch();
    return cudaGetLastError();
}

template <int V, int NT, class Loc, bool LAB = false>
static cudaError_t launch_repair(const Loc &loc, uint32_t ntiles, uint32_t *status, cudaStream_t st,
                                 const LabelArgs &la = LabelArgs{})
{
    using VV = Variant<V>;
    using RS = RepairShape<VV::LX, VV::LY, VV::LZ>;
    cudaError_t e;
    if ((e = repair_attrs<V, NT, Loc, LAB>()) != cudaSuccess) return e;
    k_repair<VV::LX, VV::LY, VV::LZ, NT, Loc, LAB><<<ntiles, NT, LAB ? RS::kSmemLab : RS::kSmem, st>>>(loc, status,
                                                                                                   la);
    count_launch();
    return cudaGetLastError();
}

// Build steps with tile variant V and the knobs of cfg (MT_CFG_* bits of
// include/mt.h): the number of level buckets of the tile kernel (its merge
// and repair rounds) and the CTA size of the repair kernel. Every
// configuration gives the same triplets.
template <int V, class Loc>
static cudaError_t run_build(const Loc &loc, uint32_t ntiles, uint32_t *queue, int persistent_grid, bool full,
                             uint32_t *status, cudaStream_t st, uint32_t cfg, const LabelArgs *la = nullptr)
{
    using VV = Variant<V>;
    cudaError_t e;
    {
        PhaseScope ps(kTile, st);
        e = (cfg & MT_CFG_FOUR_ROUNDS)
                ? launch_tile<V, 4>(loc, ntiles, queue, persistent_grid, full, status, st)
                : launch_tile<V, kBuckets>(loc, ntiles, queue, persistent_grid, full, status, st);
        if (e != cudaSuccess) return e;
    }
    {
        PhaseScope ps(kMerge, st);
        k_cross<VV::LX, VV::LY, VV::LZ, Loc><<<ntiles, 256, 0, st>>>(loc, status);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    PhaseScope ps(kRepair, st);
    if constexpr (std::is_same<Loc, OneField>::value) {
        // a single field is repaired (and labelled) in 32 x 16 x 16 bricks
        using RV = Variant<2>;
        OneField rl = loc;
        rl.d.ntx = (loc.d.nx + (1u << RV::LX) - 1) >> RV::LX;
        rl.d.nty = (loc.d.ny + (1u << RV::LY) - 1) >> RV::LY;
        const uint32_t rn = rl.d.ntx * rl.d.nty * ((loc.d.nz + (1u << RV::LZ) - 1) >> RV::LZ);
        if (la)
            return (cfg & MT_CFG_REPAIR_256) ? launch_repair<2, 256, Loc, true>(rl, rn, status, st, *la)
                                             : launch_repair<2, 512, Loc, true>(rl, rn, status, st, *la);
        return (cfg & MT_CFG_REPAIR_256) ? launch_repair<2, 256>(rl, rn, status, st)
                                         : launch_repair<2, 512>(rl, rn, status, st);
    } else {
        return (cfg & MT_CFG_REPAIR_256) ? launch_repair<V, 256>(loc, ntiles, status, st)
                                         : launch_repair<V, 512>(loc, ntiles, status, st);
    }
}

// A single field in the tile shape of variant V (0, or 2 with MT_CFG_LARGE_TILES).
template <int V>
static cudaError_t build_one(const float *f, uint64_t *W, uint32_t nx, uint32_t ny, uint32_t nz, Workspace &ws,
                             uint32_t *faces, float sg, cudaStream_t st, uint32_t cfg, const LabelArgs *la)
{
    using VV = Variant<V>;
    OneField loc;
    loc.d = FieldDesc{};
    loc.d.f = f;
    loc.d.W = W;
    loc.d.faces = faces;
    loc.d.sg = sg;
    loc.d.nx = nx, loc.d.ny = ny, loc.d.nz = nz;
    loc.d.n = (uint64_t)nx * ny * nz;
    loc.d.ntx = (nx + (1u << VV::LX) - 1) >> VV::LX;
    loc.d.nty = (ny + (1u << VV::LY) - 1) >> VV::LY;
    const uint32_t ntz = (nz + (1u << VV::LZ) - 1) >> VV::LZ;
    const uint64_t ntiles = (uint64_t)loc.d.ntx * loc.d.nty * ntz;
    const bool full = nx % (1u << VV::LX) == 0 && ny % (1u << VV::LY) == 0 && nz % (1u << VV::LZ) == 0;
    return run_build<V>(loc, (uint32_t)ntiles, nullptr, 0, full, ws.status, st, cfg, la);
}

cudaError_t launch_build(const float *f, uint64_t *W, uint32_t nx, uint32_t ny, uint32_t nz, Workspace &ws,
                         uint32_t *faces, float sg, cudaStream_t st, uint32_t cfg, const LabelArgs *la)
{
    if (cfg & MT_CFG_LARGE_TILES) return build_one<2>(f, W, nx, ny, nz, ws, faces, sg, st, cfg, la);
    return build_one<0>(f, W, nx, ny, nz, ws, faces, sg, st, cfg, la);
}

// The tile kernel with 64-bit ids and 128-bit output words (the wide path):
// one CTA per 32x16x16 tile (the tiles whose boundaries k_w_cross merges),
// no face buffer.
cudaError_t launch_tile_wide(const float *f, uint64_t *W2, uint32_t nx, uint32_t ny, uint32_t nz, float sg,
                             uint32_t *status, cudaStream_t st)
{
    using VV = Variant<2>;
    using TS = Tile<VV::LX, VV::LY, VV::LZ, VV::NT>;
    OneField loc;
    loc.d = FieldDesc{};
    loc.d.f = f;
    loc.d.W = W2;
    loc.d.faces = nullptr;
    loc.d.sg = sg;
    loc.d.nx = nx, loc.d.ny = ny, loc.d.nz = nz;
    loc.d.n = (uint64_t)nx * ny * nz;
    loc.d.ntx = (nx + (1u << VV::LX) - 1) >> VV::LX;
    loc.d.nty = (ny + (1u << VV::LY) - 1) >> VV::LY;
    const uint64_t ntz = (nz + (1u << VV::LZ) - 1) >> VV::LZ;
    const uint64_t ntiles = (uint64_t)loc.d.ntx * loc.d.nty * ntz;
    if (ntiles >= 0x80000000ull) return cudaErrorInvalidValue;
    const bool full = nx % (1u << VV::LX) == 0 && ny % (1u << VV::LY) == 0 && nz % (1u << VV::LZ) == 0;
    static AttrFlags attr[2];
    auto kfull = k_tile<VV::LX, VV::LY, VV::LZ, VV::NT, kBuckets, OneField, true, true>;
    auto kpart = k_tile<VV::LX, VV::LY, VV::LZ, VV::NT, kBuckets, OneField, false, true>;
    auto kern = full ? kfull : kpart;
    int dev;
    if (attr[full].pending(dev)) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TS::kSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        attr[full].done(dev);
    }
    kern<<<(unsigned)ntiles, VV::NT, TS::kSmem, st>>>(loc, (uint32_t)ntiles, nullptr, status);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_batch_build(const FieldDesc *d_descs, uint32_t nfields, uint32_t ntiles, uint32_t cfg,
                               uint32_t *status, uint32_t *queue, cudaStream_t st)
{
    ManyFields loc{d_descs, nfields};
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    // persistent grid: as many CTAs as fit on the GPU at once
    const bool small = cfg & MT_CFG_SMALL_TILES;
    const int per_sm = small ? 1536 / Variant<1>::NT : 2048 / Variant<0>::NT;
    const int grid = device_sms() * per_sm;
    if (small) return run_build<1>(loc, ntiles, queue, grid, false, status, st, cfg);
    return run_build<0>(loc, ntiles, queue, grid, false, status, st, cfg);
}

}  // namespace mt
