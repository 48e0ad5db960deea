// Queries on a finished triplet merge tree:
//   k_pairs_count / k_scan_counts / k_pairs_write
//       0-dimensional persistence pairs (minimum u, saddle s) for every u with
//       W[u].s != u, in ascending u (ordered stream compaction);
//   k_labels
//       representatives at a threshold t (components of G_t).
#include <cuda_runtime.h>

#include "mt_device.cuh"
#include "mt_fields.cuh"
#include "mt_internal.h"

namespace mt {

// ------------------------------------------------------------------ pairs
//
// One CTA per chunk of kCompactChunk consecutive vertices of a field; warp w
// owns the contiguous slice [w * 512, (w + 1) * 512) of the chunk and reads it
// in 16 coalesced rows of 32. A pass counts the pairs of each chunk (and finds
// the roots), a scan per field turns the counts into offsets, and a second
// pass writes each chunk's pairs at its offset in order: every warp keeps its
// 16 triplets in registers, ranks its flags with ballots, and one barrier
// combines the 8 warp totals, which keeps the ascending order.
constexpr int kCompactThreads = 256;

// Persistence simplification (SIMP): the pair (u, s) of a branch minimum u is
// kept when its persistence f(s) - f(u), computed in float32 on the values
// the order sees (sg * f), is at least eps. Without SIMP every pair is kept
// and f is not read (a separate instantiation, so that the plain kernels
// keep their loads of all rows ahead of any use).
template <bool SIMP>
__device__ __forceinline__ bool keep_pair(const FieldDesc &fd, uint64_t T, uint32_t u, float eps)
{
    if (tri_s(T) == u) return false;
    if (!SIMP) return true;
    const float fu = fd.sg * __ldg(fd.f + u), fs = fd.sg * __ldg(fd.f + tri_s(T));
    return fs - fu >= eps;
}
constexpr int kCompactWarps = kCompactThreads / 32;
constexpr int kCompactRows = kCompactChunk / kCompactThreads;  // rows of 32 per warp
static_assert(kCompactRows * 32 * kCompactWarps == kCompactChunk, "chunk = warps x rows x 32");

template <class Loc, bool SIMP>
__global__ void __launch_bounds__(kCompactThreads) k_pairs_count(Loc loc, uint32_t *counts, float eps,
                                                                 const uint32_t *status)
{
    if (block_skips(status)) return;
    __shared__ uint32_t warp_sum[kCompactWarps];
    uint64_t local;
    uint32_t fi;
    const FieldDesc fd = loc.chunk(blockIdx.x, local, fi);
    const uint64_t *__restrict__ W = fd.W;
    const uint64_t n = fd.n;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t b0 = local * kCompactChunk + (uint64_t)warp * (kCompactRows * 32);
    uint32_t c = 0;
    // all rows are loaded before any is used, so that their loads overlap
    uint64_t Tr[kCompactRows];
#pragma unroll
    for (int r = 0; r < kCompactRows; r++) {
        const uint64_t u = b0 + (uint64_t)r * 32 + lane;
        Tr[r] = u < n ? W[u] : tri_pack((uint32_t)u, (uint32_t)u + 1);  // past the end: neither pair nor root
    }
#pragma unroll
    for (int r = 0; r < kCompactRows; r++) {
        const uint64_t u = b0 + (uint64_t)r * 32 + lane;
        const uint64_t T = Tr[r];
        if (tri_s(T) != (uint32_t)u) {
            c += keep_pair<SIMP>(fd, T, (uint32_t)u, eps);
        } else if (tri_v(T) == (uint32_t)u) {
            atomicAdd(reinterpret_cast<unsigned long long *>(fd.meta + 1), 1ull);
            fd.meta[2] = u;
        }
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) warp_sum[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t tot = 0;
        for (int w = 0; w < kCompactWarps; w++) tot += warp_sum[w];
        counts[blockIdx.x] = tot;
    }
}

// Exclusive scan of one field's chunk counts in place (one CTA of 1024
// threads per field); the field's total goes to its meta[0] and, in a batch,
// to npairs[field]. Warp w owns a contiguous range of chunks and reads it in
// coalesced rows of 32: a first pass sums the range, one warp scans the 32
// sums, and a second pass scans each row with shuffles on top of the carry.
template <class Loc>
__global__ void __launch_bounds__(1024) k_scan_counts(Loc loc, uint32_t *counts, uint64_t *npairs,
                                                      const uint32_t *status)
{
    if (block_skips(status)) return;
    __shared__ uint64_t wsum[32];
    const FieldDesc fd = loc.field(blockIdx.x);
    uint32_t *cnt = counts + fd.chunk0;
    const uint64_t m = (fd.n + kCompactChunk - 1) / kCompactChunk;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t per = ((m + 31) / 32 + 31) / 32 * 32;  // chunks per warp, whole rows
    const uint64_t a = warp * per, b = a + per < m ? a + per : m;
    uint64_t s = 0;
    for (uint64_t i = a + lane; i < b; i += 32) s += cnt[i];
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
        wsum[lane] = incl - v;  // exclusive
        if (lane == 31) {
            fd.meta[0] = incl;
            if (npairs) npairs[blockIdx.x] = incl;
        }
    }
    __syncthreads();
    uint64_t carry = wsum[warp];
    for (uint64_t r = a; r < b; r += 32) {
        const uint64_t i = r + lane;
        const uint32_t c = i < b ? cnt[i] : 0u;
        uint32_t incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        if (i < b) cnt[i] = (uint32_t)(carry + incl - c);
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
}

template <class Loc, bool SIMP>
__global__ void __launch_bounds__(kCompactThreads) k_pairs_write(Loc loc, const uint32_t *offsets, float eps,
                                                                 const uint32_t *status)
{
    if (block_skips(status)) return;
    __shared__ uint32_t warp_cnt[kCompactWarps];
    uint64_t local;
    uint32_t fi;
    const FieldDesc fd = loc.chunk(blockIdx.x, local, fi);
    const uint64_t *__restrict__ W = fd.W;
    const uint64_t n = fd.n, cap = fd.cap;
    uint32_t *pairs = fd.pairs;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t b0 = local * kCompactChunk + (uint64_t)warp * (kCompactRows * 32);
    uint64_t Tr[kCompactRows];
    uint32_t c = 0;
#pragma unroll
    for (int r = 0; r < kCompactRows; r++) {
        const uint64_t u = b0 + (uint64_t)r * 32 + lane;
        Tr[r] = u < n ? W[u] : tri_pack((uint32_t)u, (uint32_t)u);  // past the end: no pair
        c += __popc(__ballot_sync(0xffffffffu, keep_pair<SIMP>(fd, Tr[r], (uint32_t)u, eps)));
    }
    if (lane == 0) warp_cnt[warp] = c;
    __syncthreads();
    uint64_t run = offsets[blockIdx.x];
    for (uint32_t w = 0; w < warp; w++) run += warp_cnt[w];
    const uint32_t below = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kCompactRows; r++) {
        const uint64_t u = b0 + (uint64_t)r * 32 + lane;
        const bool flag = keep_pair<SIMP>(fd, Tr[r], (uint32_t)u, eps);
        const uint32_t ball = __ballot_sync(0xffffffffu, flag);
        if (flag) {
            const uint64_t pos = run + __popc(ball & below);
            if (pos < cap) {
                pairs[2 * pos] = (uint32_t)u;
                pairs[2 * pos + 1] = tri_s(Tr[r]);
            }
        }
        run += __popc(ball);
    }
}

template <class Loc>
static cudaError_t run_pairs(const Loc &loc, uint32_t nfields, uint64_t nchunks, uint32_t *counts, uint64_t *npairs,
                             const uint32_t *status, cudaStream_t st, float eps = 0.0f)
{
    PhaseScope ps(kPairs, st);
    count_launch(3);
    const bool simp = eps > 0.0f;
    if (simp) k_pairs_count<Loc, true><<<(unsigned)nchunks, kCompactThreads, 0, st>>>(loc, counts, eps, status);
    else k_pairs_count<Loc, false><<<(unsigned)nchunks, kCompactThreads, 0, st>>>(loc, counts, eps, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_scan_counts<Loc><<<nfields, 1024, 0, st>>>(loc, counts, npairs, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (simp) k_pairs_write<Loc, true><<<(unsigned)nchunks, kCompactThreads, 0, st>>>(loc, counts, eps, status);
    else k_pairs_write<Loc, false><<<(unsigned)nchunks, kCompactThreads, 0, st>>>(loc, counts, eps, status);
    return cudaGetLastError();
}

cudaError_t launch_pairs(const uint64_t *W, uint64_t n, uint32_t *pairs, uint64_t cap, Workspace &ws,
                         cudaStream_t st, const float *f, float sg, float eps)
{
    cudaError_t e = cudaMemsetAsync(ws.meta, 0, 3 * sizeof(uint64_t), st);
    if (e != cudaSuccess) return e;
    OneField loc;
    loc.d = FieldDesc{};
    loc.d.W = const_cast<uint64_t *>(W);
    loc.d.pairs = pairs;
    loc.d.meta = ws.meta;
    loc.d.n = n;
    loc.d.cap = cap;
    loc.d.f = f;
    loc.d.sg = sg;
    return run_pairs(loc, 1, ws.nchunks, ws.counts, nullptr, ws.status, st, eps);
}

cudaError_t launch_batch_pairs(const FieldDesc *d_descs, uint32_t nfields, uint64_t nchunks, uint32_t *counts,
                               uint64_t *npairs, const uint32_t *status, cudaStream_t st)
{
    ManyFields loc{d_descs, nfields};
    return run_pairs(loc, nfields, nchunks, counts, npairs, status, st);
}

// ----------------------------------------------------------------- labels
//
// Components of G_t = {u : f[u] <= t} (Section 2.1): the label of u is its
// representative at level t (Algorithm 4 with the value test f(s) <= t that
// the paper's Representative uses), the deepest vertex of u's component, or
// 0xFFFFFFFF when f[u] > t. An inner vertex u with f[u] <= t hops to its
// deepest vertex v first (its link's saddle is u itself); the chain of branch
// links is then followed while their saddles lie in G_t.
//
// One CTA per brick of 32 x 16 x 16 vertices, in three steps: every vertex in
// G_t enters the start of its chain (its target v, or u itself for a minimum
// or a root) in a shared-memory hash and keeps the slot; the chain of every
// hashed start is followed once; every vertex then takes its label from its
// slot. The vertices of a brick share a few hundred starts, so each vertex
// costs one read of f and W and one write, and the chases run once per start.
// A vertex whose start finds no room in the hash follows its chain itself.
//
// With eps > 0 the labels are those of the simplified field in which every
// branch of persistence below eps is filled up to its saddle: a component of
// G_t whose representative r heads such a branch (r not the root, f(s) - f(r)
// < eps in float32 for r's saddle s) lies inside a filled pit and leaves G_t,
// its vertices labelled 0xFFFFFFFF. No other component changes: by the elder
// rule a branch is never less persistent than one that merges into it, so a
// long branch never lies inside a short one's pit.
constexpr uint32_t kLabLX = 5, kLabLY = 4, kLabLZ = 4;
constexpr uint32_t kLabThreads = 512;
constexpr uint32_t kLabHashLog = kLabelHashLog;  // 4096 slots (64 in a stress build)
constexpr size_t kLabSmem = ((size_t)8 << kLabHashLog) + ((size_t)2 << (kLabLX + kLabLY + kLabLZ));

__global__ void __launch_bounds__(kLabThreads, 4) k_labels(const Field f, const uint64_t *__restrict__ W, uint32_t nx,
                                                           uint32_t ny, uint32_t nz, uint32_t ntx, uint32_t nty,
                                                           float t, float eps, uint32_t *__restrict__ labels,
                                                           uint32_t *status)
{
    const uint32_t n = nx * ny * nz;
    const uint32_t limit = n < kChaseLimit ? n : kChaseLimit;
    if (block_skips(status)) return;
    constexpr uint32_t TX = 1u << kLabLX, TY = 1u << kLabLY, TZ = 1u << kLabLZ, TV = TX * TY * TZ;
    constexpr uint32_t HS = 1u << kLabHashLog, NT = kLabThreads, NB = 4;
    constexpr uint32_t EMPTY = 0xFFFFFFFFu, kProbes = 16;
    constexpr uint16_t OUT = 0xFFFFu, SELF = 0xFFFEu;  // slot codes: not in G_t; no room in the hash
    static_assert(HS <= SELF && TV % (NT * NB) == 0, "slot codes and batches");
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *hkey = smem;               // chain starts
    uint32_t *hval = hkey + HS;          // their representatives at t
    uint16_t *vslot = reinterpret_cast<uint16_t *>(hval + HS);  // per vertex: slot or code
    const unsigned long long *Wq = reinterpret_cast<const unsigned long long *>(W);

    const uint32_t tile = blockIdx.x;
    const uint32_t tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
    const uint32_t x0 = tx * TX, y0 = ty * TY, z0 = tz * TZ;
    const uint32_t wx = min(TX, nx - x0), wy = min(TY, ny - y0), wz = min(TZ, nz - z0);
    const uint32_t nxy = nx * ny;
    const uint32_t base = z0 * nxy + y0 * nx + x0;
    auto gid_of = [&](uint32_t l) {
        return base + (l >> (kLabLX + kLabLY)) * nxy + ((l >> kLabLX) & (TY - 1)) * nx + (l & (TX - 1));
    };
    auto inside = [&](uint32_t l) {
        return (l & (TX - 1)) < wx && ((l >> kLabLX) & (TY - 1)) < wy && (l >> (kLabLX + kLabLY)) < wz;
    };
    // representative at t of the chain from x: the caller's triplets are
    // followed only through ids < n, and for at most `limit` links (a chain
    // of a valid tree is shorter than n, so a longer one means a cycle)
    bool ok = true, bad = false;
    auto chase = [&](uint32_t x) -> uint32_t {
        for (uint32_t h = 0;; h++) {
            const uint64_t T = __ldg(Wq + x);
            const uint32_t s = tri_s(T);
            if (T == tri_pack(x, x)) return x;
            if (s >= n || tri_v(T) >= n) {
                bad = true;
                return x;
            }
            if (!(f[s] <= t)) return x;
            x = tri_v(T);
            if (h >= limit) {
                ok = false;
                return x;
            }
        }
    };
    // the representative, or 0xFFFFFFFF if it heads a branch shorter than eps
    auto simplified = [&](uint32_t r) -> uint32_t {
        if (!(eps > 0.0f)) return r;
        const uint64_t T = __ldg(Wq + r);
        const uint32_t s = tri_s(T);
        if (s == r || s >= n) return r;  // the root (or an inner vertex of a corrupt tree)
        return f[s] - f[r] >= eps ? r : 0xFFFFFFFFu;
    };

    for (uint32_t i = threadIdx.x; i < HS; i += NT) hkey[i] = EMPTY;
    __syncthreads();

    // 1. chain starts into the hash
    volatile uint32_t *vhk = hkey;
    for (uint32_t l0 = 0; l0 < TV; l0 += NT * NB) {
        uint64_t Tb[NB];
        float fb[NB];
#pragma unroll
        for (uint32_t k = 0; k < NB; k++) {
            const uint32_t l = l0 + k * NT + threadIdx.x;
            const uint32_t u = gid_of(l);
            const bool in = inside(l);
            fb[k] = in ? f[u] : 0.0f;
            Tb[k] = in ? __ldg(Wq + u) : tri_pack(u, u);
        }
#pragma unroll
        for (uint32_t k = 0; k < NB; k++) {
            const uint32_t l = l0 + k * NT + threadIdx.x;
            if (!inside(l)) continue;
            const uint32_t u = gid_of(l);
            if (!(fb[k] <= t)) {
                vslot[l] = OUT;
                continue;
            }
            const uint32_t s = tri_s(Tb[k]), v = tri_v(Tb[k]);
            if (s >= n || v >= n) {  // leave it to the vertex's own chase, which reports it
                vslot[l] = SELF;
                continue;
            }
            const uint32_t st = (s == u && v != u) ? v : u;
            uint32_t h = (st * 0x9E3779B1u) >> (32 - kLabHashLog);
            uint16_t slot = SELF;
            for (uint32_t p = 0; p < kProbes; p++) {
                uint32_t kk = vhk[h];
                if (kk == EMPTY) kk = atomicCAS(hkey + h, EMPTY, st);
                if (kk == EMPTY || kk == st) {
                    slot = (uint16_t)h;
                    break;
                }
                h = (h + 1) & (HS - 1);
            }
            vslot[l] = slot;
        }
    }
    __syncthreads();

    // 2. one chase per hashed start. Each warp takes the occupied slots of
    //    its own HS / warps slots and deals them out to its lanes in order
    //    (ballot masks in registers), so that every lane has a chase instead
    //    of one lane per fixed group of mostly empty slots.
    constexpr uint32_t PER = HS / (NT / 32);  // slots per warp
    if constexpr (PER >= 32 && PER % 32 == 0) {
        constexpr uint32_t G = PER >= 32 ? PER / 32 : 1;  // (1 only in the branch not taken)
        const uint32_t lane = threadIdx.x & 31, wbase = (threadIdx.x >> 5) * PER;
        uint32_t mask[G], tot = 0;
#pragma unroll
        for (uint32_t g = 0; g < G; g++) {
            mask[g] = __ballot_sync(0xffffffffu, hkey[wbase + g * 32 + lane] != EMPTY);
            tot += __popc(mask[g]);
        }
        for (uint32_t r = lane; r < tot; r += 32) {
            // the slot of rank r among the warp's occupied slots
            uint32_t rr = r, i = 0;
#pragma unroll
            for (uint32_t g = 0; g < G; g++) {
                const uint32_t c = __popc(mask[g]);
                if (rr < c && i == 0) {
                    uint32_t m = mask[g];
                    for (uint32_t k = 0; k < rr; k++) m &= m - 1;
                    i = wbase + g * 32 + __ffs(m);  // 1 + the slot
                }
                rr = rr < c ? rr : rr - c;
            }
            hval[i - 1] = simplified(chase(hkey[i - 1]));
        }
    } else {
        for (uint32_t i = threadIdx.x; i < HS; i += NT) {
            const uint32_t st = hkey[i];
            if (st != EMPTY) hval[i] = simplified(chase(st));
        }
    }
    __syncthreads();

    // 3. labels
    for (uint32_t l = threadIdx.x; l < TV; l += NT) {
        if (!inside(l)) continue;
        const uint32_t u = gid_of(l);
        const uint16_t c = vslot[l];
        labels[u] = c == OUT ? 0xFFFFFFFFu : c == SELF ? simplified(chase(u)) : hval[c];
    }
    if (!ok) raise_status(status, ST_TIMEOUT);
    if (bad) raise_status(status, ST_CORRUPT);
}

cudaError_t launch_labels(const float *f, const uint64_t *W, uint32_t nx, uint32_t ny, uint32_t nz, float t,
                          float sg, uint32_t *labels, Workspace &ws, cudaStream_t st, float eps)
{
    PhaseScope ps(kLabels, st);
    count_launch();
    const uint32_t ntx = (nx + 31) >> kLabLX, nty = (ny + 15) >> kLabLY, ntz = (nz + 15) >> kLabLZ;
    static AttrFlags attr;
    int dev;
    if (attr.pending(dev)) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_labels, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLabSmem);
        if (e != cudaSuccess) return e;
        attr.done(dev);
    }
    k_labels<<<ntx * nty * ntz, kLabThreads, kLabSmem, st>>>(Field{f, sg}, W, nx, ny, nz, ntx, nty, t, eps,
                                                            labels, ws.status);
    return cudaGetLastError();
}

}  // namespace mt
