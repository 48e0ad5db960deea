// Branch decomposition of a finished triplet merge tree.
//
// Every vertex belongs to one branch of the tree (Section 2.1): a minimum u
// (W[u].s != u, or the root W[u] = (u, u)) heads its own branch, and an inner
// vertex u (W[u] = (u, v), v != u) lies on the branch of v, the deepest
// vertex of its component at level f(u), whose minimum the arc through u
// descends to. The call lists all vertices grouped by branch -- branches by
// ascending id of their minimum, each group in the vertex order (value, then
// index), so that it starts with its minimum -- and the offset of every group:
// the per-branch vertex lists that the CPU implementation keeps beside its
// triplets (Section 3.1), as one array.
//
// The grouping is a stable least-significant-digit radix sort of 64-bit keys
// (branch << 32) | order key of f, with vertex ids as values, 8 bits per
// pass; passes whose digit is the same in every key are skipped. A pass is a
// per-block digit histogram, an exclusive scan of the histograms (digit
// major, block minor), and a scatter that ranks each block's keys stably: a
// warp owns a contiguous run of the block's keys, finds the lanes sharing a
// digit with eight ballots, and adds the counts of earlier warps and earlier
// rounds. Group heads are then compacted into the offsets.
#include <cuda_runtime.h>

#include "../../include/mt.h"
#include "mt_device.cuh"
#include "mt_internal.h"

namespace mt {

mt_status status_from_bits(uint32_t bits);  // mt_api.cu

constexpr uint32_t kSortThreads = 256;
constexpr uint32_t kSortWarps = kSortThreads / 32;
constexpr uint32_t kSortRows = 8;                                   // keys per thread
constexpr uint32_t kSortBlock = kSortThreads * kSortRows;           // keys per block
constexpr uint32_t kScanItems = 4096;                               // entries per scan block

// order key of a float: unsigned order = float order, -0 and +0 equal
__device__ __forceinline__ uint32_t okey(float x)
{
    const uint32_t b = x == 0.0f ? 0u : __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// keys[u] = (branch(u) << 32) | okey(sg * f[u]); vals[u] = u; the OR and AND
// of all keys tell which digits vary
__global__ void __launch_bounds__(256) k_branch_keys(const Field f, const uint64_t *__restrict__ W, uint32_t n,
                                                     uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                                                     unsigned long long *orand, uint32_t *status)
{
    unsigned long long o = 0, a = ~0ull;
    bool bad = false;
    // 64-bit index: near n = 2^32 a 32-bit index plus the stride would wrap
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t u = (uint32_t)i;
        const uint64_t T = W[u];
        const uint32_t s = tri_s(T), v = tri_v(T);
        if (s >= n || v >= n) bad = true;
        const uint32_t b = (s == u && v != u) ? v : u;
        const uint64_t k = ((uint64_t)b << 32) | okey(f[u]);
        keys[u] = k;
        vals[u] = u;
        o |= k;
        a &= k;
    }
    for (int d = 16; d > 0; d >>= 1) {
        o |= __shfl_xor_sync(0xffffffffu, o, d);
        a &= __shfl_xor_sync(0xffffffffu, a, d);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicOr(orand, o);
        atomicAnd(orand + 1, a);
    }
    if (bad) raise_status(status, ST_CORRUPT);
}

// hist[d * nblocks + b] = keys of block b with digit d
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint64_t *__restrict__ keys, uint32_t n,
                                                             uint32_t shift, uint32_t nblocks,
                                                             uint32_t *__restrict__ hist)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t b0 = (uint64_t)blockIdx.x * kSortBlock;
#pragma unroll
    for (uint32_t r = 0; r < kSortRows; r++) {
        const uint64_t i = b0 + r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(uint64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of m entries in three steps: per-block sums, a scan of the
// sums by one CTA, and per-block scans with the block's offset.
__global__ void __launch_bounds__(1024) k_scan_sums(const uint32_t *__restrict__ a, uint64_t m,
                                                    uint32_t *__restrict__ sums)
{
    __shared__ uint32_t part[32];
    const uint64_t b0 = (uint64_t)blockIdx.x * kScanItems;
    uint32_t s = 0;
    for (uint32_t i = threadIdx.x; i < kScanItems; i += 1024)
        if (b0 + i < m) s += a[b0 + i];
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = part[threadIdx.x];
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        if (threadIdx.x == 0) sums[blockIdx.x] = s;
    }
}

// block-wide exclusive scan of one value per thread (1024 threads)
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *part, uint32_t &total)
{
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = v;
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= (uint32_t)d) incl += y;
    }
    if (lane == 31) part[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint32_t p = part[lane], q = p;
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, q, d);
            if (lane >= (uint32_t)d) q += y;
        }
        part[lane] = q - p;
        if (lane == 31) part[32] = q;
    }
    __syncthreads();
    total = part[32];
    const uint32_t r = part[w] + incl - v;
    __syncthreads();
    return r;
}

// one CTA: sums[0..k) -> exclusive prefix in place (k <= 1024 * 64)
__global__ void __launch_bounds__(1024) k_scan_top(uint32_t *sums, uint32_t k)
{
    __shared__ uint32_t part[33];
    const uint32_t per = (k + 1023) / 1024;
    const uint32_t a = threadIdx.x * per, b = min(a + per, k);
    uint32_t s = 0;
    for (uint32_t i = a; i < b; i++) s += sums[i];
    uint32_t total;
    uint32_t run = block_excl_scan(s, part, total);
    for (uint32_t i = a; i < b; i++) {
        const uint32_t c = sums[i];
        sums[i] = run;
        run += c;
    }
}

__global__ void __launch_bounds__(1024) k_scan_apply(uint32_t *a, uint64_t m, const uint32_t *__restrict__ sums)
{
    __shared__ uint32_t part[33];
    constexpr uint32_t per = kScanItems / 1024;
    const uint64_t b0 = (uint64_t)blockIdx.x * kScanItems + (uint64_t)threadIdx.x * per;
    uint32_t v[per], s = 0;
#pragma unroll
    for (uint32_t i = 0; i < per; i++) {
        v[i] = b0 + i < m ? a[b0 + i] : 0u;
        s += v[i];
    }
    uint32_t total;
    uint32_t run = sums[blockIdx.x] + block_excl_scan(s, part, total);
#pragma unroll
    for (uint32_t i = 0; i < per; i++) {
        if (b0 + i < m) a[b0 + i] = run;
        run += v[i];
    }
}

// Stable scatter of block b's keys and values to the scanned offsets. Warp w
// owns keys [w * 256, (w + 1) * 256) of the block, read in kSortRows rounds of
// 32; a key's place within the block's run of its digit is the number of keys
// with that digit in earlier warps, in earlier rounds of its warp and on lower
// lanes of its round. The keys are first placed in shared memory in that
// order (digit by digit), then written out in order, so that consecutive
// threads write consecutive addresses of a digit's run.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint64_t *__restrict__ kin,
                                                                const uint32_t *__restrict__ vin,
                                                                uint64_t *__restrict__ kout,
                                                                uint32_t *__restrict__ vout, uint32_t n,
                                                                uint32_t shift, uint32_t nblocks,
                                                                const uint32_t *__restrict__ offs)
{
    __shared__ uint32_t cnt[kSortWarps][256];  // per-warp digit counts, then running local places
    __shared__ uint32_t base[256], lstart[256], wtot[kSortWarps];
    __shared__ uint64_t skey[kSortBlock];
    __shared__ uint32_t sval[kSortBlock];
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (uint32_t i = threadIdx.x; i < kSortWarps * 256; i += kSortThreads) (&cnt[0][0])[i] = 0;
    base[threadIdx.x] = offs[(uint64_t)threadIdx.x * nblocks + blockIdx.x];
    __syncthreads();
    const uint64_t blk0 = (uint64_t)blockIdx.x * kSortBlock;
    const uint64_t b0 = blk0 + (uint64_t)w * (kSortRows * 32);
    uint64_t k[kSortRows];
    uint32_t v[kSortRows], peers[kSortRows];
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (uint32_t r = 0; r < kSortRows; r++) {
        const uint64_t i = b0 + r * 32 + lane;
        const bool in = i < n;
        k[r] = in ? kin[i] : ~0ull;
        v[r] = in ? vin[i] : 0u;
        const uint32_t d = (uint32_t)(k[r] >> shift) & 255u;
        uint32_t p = __ballot_sync(0xffffffffu, in);
#pragma unroll
        for (uint32_t bit = 0; bit < 8; bit++) {
            const uint32_t bb = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
            p &= ((d >> bit) & 1u) ? bb : ~bb;
        }
        peers[r] = in ? p : 0u;
        if (in && (p & lt) == 0) cnt[w][d] += __popc(p);  // the group's lowest lane
        __syncwarp();
    }
    __syncthreads();
    // thread = digit: the block's count of the digit, its local start
    // (exclusive scan over digits), and the running places of the warps
    {
        const uint32_t d = threadIdx.x;
        uint32_t tot = 0;
        for (uint32_t q = 0; q < kSortWarps; q++) tot += cnt[q][d];
        uint32_t incl = tot;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        if (lane == 31) wtot[w] = incl;
        __syncthreads();
        uint32_t run = incl - tot;
        for (uint32_t q = 0; q < w; q++) run += wtot[q];
        lstart[d] = run;
        for (uint32_t q = 0; q < kSortWarps; q++) {
            const uint32_t c = cnt[q][d];
            cnt[q][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (uint32_t r = 0; r < kSortRows; r++) {
        const uint32_t p = peers[r];
        const uint32_t d = (uint32_t)(k[r] >> shift) & 255u;
        uint32_t pos = 0;
        if (p) pos = cnt[w][d] + __popc(p & lt);
        __syncwarp();
        if (p && (p & lt) == 0) cnt[w][d] += __popc(p);
        __syncwarp();
        if (p) {
            skey[pos] = k[r];
            sval[pos] = v[r];
        }
    }
    __syncthreads();
    const uint32_t valid = n - blk0 < kSortBlock ? (uint32_t)(n - blk0) : kSortBlock;
    for (uint32_t j = threadIdx.x; j < valid; j += kSortThreads) {
        const uint64_t key = skey[j];
        const uint32_t d = (uint32_t)(key >> shift) & 255u;
        const uint32_t pos = base[d] + (j - lstart[d]);
        kout[pos] = key;
        vout[pos] = sval[j];
    }
}

// group heads: position i starts a group if its branch differs from i - 1's
__global__ void __launch_bounds__(256) k_heads_count(const uint64_t *__restrict__ keys, uint32_t n,
                                                     uint32_t *__restrict__ counts)
{
    __shared__ uint32_t part[8];
    const uint64_t b0 = (uint64_t)blockIdx.x * kScanItems;
    uint32_t c = 0;
    for (uint32_t j = threadIdx.x; j < kScanItems; j += 256) {
        const uint64_t i = b0 + j;
        if (i < n) c += i == 0 || (keys[i] >> 32) != (keys[i - 1] >> 32);
    }
    for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int q = 0; q < 8; q++) t += part[q];
        counts[blockIdx.x] = t;
    }
}

// offsets[rank of the head] = its position, in order (warp w owns a
// contiguous slice of the block; ballots rank the heads of a row)
__global__ void __launch_bounds__(256) k_heads_write(const uint64_t *__restrict__ keys, uint32_t n,
                                                     const uint32_t *__restrict__ starts, uint32_t *offsets,
                                                     uint64_t cap)
{
    __shared__ uint32_t wsum[8];
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr uint32_t per = kScanItems / 8;  // keys per warp
    const uint64_t b0 = (uint64_t)blockIdx.x * kScanItems + (uint64_t)w * per;
    uint32_t c = 0;
    for (uint32_t r = 0; r < per; r += 32) {
        const uint64_t i = b0 + r + lane;
        const bool h = i < n && (i == 0 || (keys[i] >> 32) != (keys[i - 1] >> 32));
        c += __popc(__ballot_sync(0xffffffffu, h));
    }
    if (lane == 0) wsum[w] = c;
    __syncthreads();
    uint64_t run = starts[blockIdx.x];
    for (uint32_t q = 0; q < w; q++) run += wsum[q];
    for (uint32_t r = 0; r < per; r += 32) {
        const uint64_t i = b0 + r + lane;
        const bool h = i < n && (i == 0 || (keys[i] >> 32) != (keys[i - 1] >> 32));
        const uint32_t bal = __ballot_sync(0xffffffffu, h);
        if (h) {
            const uint64_t pos = run + __popc(bal & ((1u << lane) - 1u));
            if (pos < cap) offsets[pos] = (uint32_t)i;
        }
        run += __popc(bal);
    }
}

// Workspace of the branch decomposition: the common part, then two key
// arrays, one value array, the digit histograms and the scan's block sums.
struct BranchWs {
    uint64_t *k0, *k1;
    uint32_t *v1, *hist, *sums;
    unsigned long long *orand;
    uint64_t nblocks, nhist, nsums;
};

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

static size_t branch_ws(uint64_t n, BranchWs *bw, char *base)
{
    const uint64_t nblocks = (n + kSortBlock - 1) / kSortBlock;
    const uint64_t nhist = 256 * nblocks;
    const uint64_t nheads = (n + kScanItems - 1) / kScanItems;
    const uint64_t nsums = ((nhist > nheads ? nhist : nheads) + kScanItems - 1) / kScanItems;
    size_t off = a256(workspace_bytes(n));
    const size_t ok0 = off;
    off += a256(n * 8);
    const size_t ok1 = off;
    off += a256(n * 8);
    const size_t ov1 = off;
    off += a256(n * 4);
    const size_t oh = off;
    off += a256((nhist > nheads ? nhist : nheads) * 4);
    const size_t os = off;
    off += a256(nsums * 4);
    const size_t oo = off;
    off += 256;
    if (bw && base) {
        bw->k0 = reinterpret_cast<uint64_t *>(base + ok0);
        bw->k1 = reinterpret_cast<uint64_t *>(base + ok1);
        bw->v1 = reinterpret_cast<uint32_t *>(base + ov1);
        bw->hist = reinterpret_cast<uint32_t *>(base + oh);
        bw->sums = reinterpret_cast<uint32_t *>(base + os);
        bw->orand = reinterpret_cast<unsigned long long *>(base + oo);
        bw->nblocks = nblocks;
        bw->nhist = nhist;
        bw->nsums = nsums;
    }
    return off;
}

static cudaError_t scan_excl(uint32_t *a, uint64_t m, uint32_t *sums, cudaStream_t st)
{
    const uint64_t nb = (m + kScanItems - 1) / kScanItems;
    k_scan_sums<<<(unsigned)nb, 1024, 0, st>>>(a, m, sums);
    k_scan_top<<<1, 1024, 0, st>>>(sums, (uint32_t)nb);
    k_scan_apply<<<(unsigned)nb, 1024, 0, st>>>(a, m, sums);
    count_launch(3);
    return cudaGetLastError();
}

}  // namespace mt

using namespace mt;

extern "C" {

size_t mt_branches_workspace_bytes(mt_grid g)
{
    const uint64_t n = (uint64_t)g.nx * g.ny * g.nz;
    if (!g.nx || !g.ny || !g.nz || n >= 0xFFFFFFFFull) return 0;
    return branch_ws(n, nullptr, nullptr);
}

mt_status mt_branch_decomposition(const float *d_f, const uint64_t *d_W, mt_grid g, uint32_t flags, uint32_t *d_order,
                                  uint32_t *d_offsets, uint64_t offsets_cap, uint64_t *h_nbranches, void *d_ws,
                                  size_t ws_bytes, void *stream)
{
    const uint64_t n = (uint64_t)g.nx * g.ny * g.nz;
    if (!g.nx || !g.ny || !g.nz) return MT_ERR_INVALID;
    if (n >= 0xFFFFFFFFull) return MT_ERR_TOO_LARGE;
    if (!d_f || !d_W || !d_order || !h_nbranches || (offsets_cap && !d_offsets) || ((uintptr_t)d_f & 3) ||
        ((uintptr_t)d_W & 7) || ((uintptr_t)d_order & 3) || ((uintptr_t)d_offsets & 3) || (flags & ~MT_SUPERLEVEL))
        return MT_ERR_INVALID;
    Workspace ws;
    if (ws_bytes < branch_ws(n, nullptr, nullptr) || !carve_workspace(d_ws, ws_bytes, n, ws)) return MT_ERR_INVALID;
    BranchWs bw;
    branch_ws(n, &bw, static_cast<char *>(d_ws));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float sg = (flags & MT_SUPERLEVEL) ? -1.0f : 1.0f;
    const unsigned long long init[2] = {0ull, ~0ull};
    PhaseScope ps(kBranches, st);
    if (cudaMemcpyAsync(bw.orand, init, sizeof(init), cudaMemcpyHostToDevice, st) != cudaSuccess) return MT_ERR_CUDA;
    // the 64-bit keys go to k0 and the values to d_order; every pass swaps
    const uint64_t kmax = (uint64_t)device_sms() * 16;  // grid-stride: 16 CTAs of 256 per SM
    const unsigned kgrid = (unsigned)((n + 255) / 256 < kmax ? (n + 255) / 256 : kmax);
    k_branch_keys<<<kgrid, 256, 0, st>>>(Field{d_f, sg}, d_W, (uint32_t)n, bw.k0, d_order, bw.orand, ws.status);
    count_launch();
    unsigned long long orand[2];
    uint32_t bits = 0;
    if (cudaMemcpyAsync(orand, bw.orand, sizeof(orand), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&bits, ws.status, sizeof(bits), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return MT_ERR_CUDA;
    if (bits) return status_from_bits(bits);
    const unsigned long long vary = orand[0] ^ orand[1];
    uint64_t *kin = bw.k0, *kout = bw.k1;
    uint32_t *vin = d_order, *vout = bw.v1;
    for (uint32_t shift = 0; shift < 64; shift += 8) {
        if (!((vary >> shift) & 255ull)) continue;  // the same digit in every key
        k_radix_hist<<<(unsigned)bw.nblocks, kSortThreads, 0, st>>>(kin, (uint32_t)n, shift, (uint32_t)bw.nblocks,
                                                                   bw.hist);
        count_launch();
        if (scan_excl(bw.hist, bw.nhist, bw.sums, st) != cudaSuccess) return MT_ERR_CUDA;
        k_radix_scatter<<<(unsigned)bw.nblocks, kSortThreads, 0, st>>>(kin, vin, kout, vout, (uint32_t)n, shift,
                                                                      (uint32_t)bw.nblocks, bw.hist);
        count_launch();
        uint64_t *tk = kin;
        kin = kout, kout = tk;
        uint32_t *tv = vin;
        vin = vout, vout = tv;
    }
    if (vin != d_order &&
        cudaMemcpyAsync(d_order, vin, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return MT_ERR_CUDA;
    // group offsets: heads counted per block (the last block's count kept
    // aside), scanned into starts, then written in order
    const uint64_t nhb = (n + kScanItems - 1) / kScanItems;
    uint32_t *last = reinterpret_cast<uint32_t *>(bw.orand);
    k_heads_count<<<(unsigned)nhb, 256, 0, st>>>(kin, (uint32_t)n, bw.hist);
    count_launch();
    if (cudaMemcpyAsync(last, bw.hist + nhb - 1, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return MT_ERR_CUDA;
    if (scan_excl(bw.hist, nhb, bw.sums, st) != cudaSuccess) return MT_ERR_CUDA;
    k_heads_write<<<(unsigned)nhb, 256, 0, st>>>(kin, (uint32_t)n, bw.hist, d_offsets, offsets_cap);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return MT_ERR_CUDA;
    uint32_t tail[2] = {0, 0};  // start of the last block's heads, their count
    if (cudaMemcpyAsync(tail, bw.hist + nhb - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(tail + 1, last, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return MT_ERR_CUDA;
    const uint64_t nb = (uint64_t)tail[0] + tail[1];
    *h_nbranches = nb;
    if (nb + 1 > offsets_cap) return MT_ERR_CAPACITY;
    const uint32_t end = (uint32_t)n;
    if (cudaMemcpyAsync(d_offsets + nb, &end, sizeof(uint32_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return MT_ERR_CUDA;
    return MT_OK;
}

}  // extern "C"
