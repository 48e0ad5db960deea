// Kernels that build the triplet merge tree (Algorithm 1 of the paper):
//   k_init     initialisation, seeded with the lowest lower neighbour
//   k_descend  pointer jumping along the steepest-descent links
//   k_merge    Merge (Algorithm 3) of every grid edge with 64-bit CAS
//   k_repair   Repair (Algorithm 5) via Representative (Algorithm 4)
#include <cuda_runtime.h>

#include "mt_device.cuh"
#include "mt_internal.h"

namespace mt {

// ---------------------------------------------------------------- k_init
//
// Algorithm 1 starts from the tree of the graph without edges, T[u] = (u, u).
// Here every vertex u that has a neighbour before it starts from
// T[u] = (u, lln(u)) instead, lln(u) its lowest lower 6-neighbour: this is a
// valid normalised triplet of the graph that holds only the steepest-descent
// edges (lln(u) comes before u and the two are joined at level f(u)), so the
// merge phase may start from it; the descent edge itself then needs no merge.
// lln(u) is the first vertex of the closed neighbourhood {u} + N(u) in the
// vertex order, and u is a local minimum iff that first vertex is u itself.
//
// Each thread handles V consecutive x of one row (V = 4 with float4 loads
// when rows are 16-byte aligned). The stencil rows y+-1 and z+-1 are re-read
// by the neighbouring rows' threads and served from L1/L2, so HBM sees each
// value about once. Non-finite values raise ST_NONFINITE.
template <int V>
__global__ void __launch_bounds__(256) k_init(const float *__restrict__ f, uint64_t *__restrict__ W, uint32_t nx,
                                              uint32_t ny, uint32_t nz, uint32_t nxq, uint32_t nthreads,
                                              uint32_t *status)
{
    const uint64_t nxy = (uint64_t)nx * ny;
    for (uint64_t tt = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; tt < nthreads;
         tt += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t t = (uint32_t)tt;
        const uint32_t xq = t % nxq;
        const uint32_t row = t / nxq;  // y + ny * z
        const uint32_t y = row % ny, z = row / ny;
        const uint32_t x0 = xq * V;
        const uint64_t base = (uint64_t)row * nx + x0;
        float c[V], ym[V], yp[V], zm[V], zp[V];
        if constexpr (V == 4) {
            const float4 cc = __ldg(reinterpret_cast<const float4 *>(f + base));
            c[0] = cc.x, c[1] = cc.y, c[2] = cc.z, c[3] = cc.w;
            if (y > 0) {
                const float4 q = __ldg(reinterpret_cast<const float4 *>(f + base - nx));
                ym[0] = q.x, ym[1] = q.y, ym[2] = q.z, ym[3] = q.w;
            }
            if (y + 1 < ny) {
                const float4 q = __ldg(reinterpret_cast<const float4 *>(f + base + nx));
                yp[0] = q.x, yp[1] = q.y, yp[2] = q.z, yp[3] = q.w;
            }
            if (z > 0) {
                const float4 q = __ldg(reinterpret_cast<const float4 *>(f + base - nxy));
                zm[0] = q.x, zm[1] = q.y, zm[2] = q.z, zm[3] = q.w;
            }
            if (z + 1 < nz) {
                const float4 q = __ldg(reinterpret_cast<const float4 *>(f + base + nxy));
                zp[0] = q.x, zp[1] = q.y, zp[2] = q.z, zp[3] = q.w;
            }
        } else {
            c[0] = __ldg(f + base);
            if (y > 0) ym[0] = __ldg(f + base - nx);
            if (y + 1 < ny) yp[0] = __ldg(f + base + nx);
            if (z > 0) zm[0] = __ldg(f + base - nxy);
            if (z + 1 < nz) zp[0] = __ldg(f + base + nxy);
        }
        const float xl = x0 > 0 ? __ldg(f + base - 1) : 0.f;
        const float xr = x0 + V < nx ? __ldg(f + base + V) : 0.f;
        uint64_t out[V];
#pragma unroll
        for (int j = 0; j < V; j++) {
            const uint32_t x = x0 + j;
            const uint32_t u = (uint32_t)(base + j);
            float fb = c[j];
            uint32_t b = u;
            if (!isfinite(fb)) raise_status(status, ST_NONFINITE);
            // candidates in ascending index order; `before` settles ties
            if (z > 0 && before(zm[j], u - (uint32_t)nxy, fb, b)) fb = zm[j], b = u - (uint32_t)nxy;
            if (y > 0 && before(ym[j], u - nx, fb, b)) fb = ym[j], b = u - nx;
            if (x > 0) {
                const float w = j > 0 ? c[j - 1] : xl;
                if (before(w, u - 1, fb, b)) fb = w, b = u - 1;
            }
            if (x + 1 < nx) {
                const float w = j + 1 < V ? c[j + 1] : xr;
                if (before(w, u + 1, fb, b)) fb = w, b = u + 1;
            }
            if (y + 1 < ny && before(yp[j], u + nx, fb, b)) fb = yp[j], b = u + nx;
            if (z + 1 < nz && before(zp[j], u + (uint32_t)nxy, fb, b)) fb = zp[j], b = u + (uint32_t)nxy;
            out[j] = tri_pack(u, b);
        }
        if constexpr (V == 4) {
            ulonglong2 *dst = reinterpret_cast<ulonglong2 *>(W + base);
            dst[0] = make_ulonglong2(out[0], out[1]);
            dst[1] = make_ulonglong2(out[2], out[3]);
        } else {
            W[base] = out[0];
        }
    }
}

// ------------------------------------------------------------- k_descend
//
// Pointer jumping along the descent links: every vertex inside a branch,
// T[u] = (u, v), moves v down the chain of such links towards the minimum
// that steepest descent reaches, T[u] = (u, m(u)). Each replacement keeps a
// valid triplet (m(u) comes before u and is joined to it below f(u)), and
// concurrent replacements only shorten chains, so threads may read entries
// that others are rewriting. A thread takes at most `hops` steps per round;
// if any thread stopped early *more is set and the host runs another round
// (each round multiplies the jump length, so the rounds are logarithmic).
__global__ void __launch_bounds__(256) k_descend(uint64_t *W, uint64_t n, uint32_t hops, uint32_t *more,
                                                 const uint32_t *status)
{
    if (*status) return;
    bool unfinished = false;
    for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < n; u += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t T = ld_tri(W + u);
        if (tri_s(T) != (uint32_t)u || tri_v(T) == (uint32_t)u) continue;  // a minimum
        uint32_t x = tri_v(T);
        uint32_t h = 0;
        for (;;) {
            const uint64_t Tx = ld_tri(W + x);
            if (tri_s(Tx) != x || tri_v(Tx) == x) break;  // x is a minimum
            x = tri_v(Tx);
            if (++h == hops) {
                unfinished = true;
                break;
            }
        }
        if (x != tri_v(T)) st_tri(W + u, tri_pack((uint32_t)u, x));
    }
    if (unfinished) *more = 1u;
}

// ---------------------------------------------------------------- k_merge
//
// The edge loop of Algorithm 1. Thread u takes the edges to its +x, +y, +z
// neighbours. For an edge (a, b) with upper end S (the later of the two in
// the vertex order), Algorithm 1 calls Merge(S, S, lower end). After
// k_descend both ends point at their descent minima, which are joined to
// them below S, so the merge starts from those minima; if the two minima
// coincide the edge is already represented and is skipped (this covers the
// descent seed edges). Inner-branch entries are never CAS targets (a merge
// at level S only moves vertices that are deepest below S), so they stay
// stable while this kernel runs and can be read once up front.
__device__ __forceinline__ uint32_t descent_root(uint64_t T, uint32_t x)
{
    return (tri_s(T) == x && tri_v(T) != x) ? tri_v(T) : x;
}

__global__ void __launch_bounds__(256) k_merge(uint64_t *W, const float *__restrict__ f, uint32_t nx, uint32_t ny,
                                               uint32_t nz, uint64_t n, uint32_t *status)
{
    if (*status) return;
    const uint32_t nxy = nx * ny;
    for (uint64_t uu = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; uu < n;
         uu += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t u = (uint32_t)uu;
        const uint32_t x = u % nx, y = (u / nx) % ny, z = u / nxy;
        const float fu = __ldg(f + u);
        const uint32_t du = descent_root(ld_tri(W + u), u);
        uint32_t nb[3];
        int k = 0;
        if (x + 1 < nx) nb[k++] = u + 1;
        if (y + 1 < ny) nb[k++] = u + nx;
        if (z + 1 < nz) nb[k++] = u + nxy;
        for (int j = 0; j < k; j++) {
            const uint32_t w = nb[j];
            const uint32_t dw = descent_root(ld_tri(W + w), w);
            if (dw == du) continue;
            const uint32_t S = before(__ldg(f + w), w, fu, u) ? u : w;
            if (!merge(W, f, S, du, dw)) raise_status(status, ST_TIMEOUT);
        }
    }
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
__global__ void __launch_bounds__(256) k_repair(uint64_t *W, const float *__restrict__ f, uint64_t n, int mode,
                                                uint32_t *status)
{
    if (*status) return;
    for (uint64_t uu = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; uu < n;
         uu += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t u = (uint32_t)uu;
        const uint64_t T = ld_tri(W + u);
        const uint32_t s = tri_s(T), t = tri_v(T);
        if (mode == 0 ? (s == u) : (s != u || t == u)) continue;
        uint32_t steps = 0;
        const uint32_t r = representative(W, f, t, s, __ldg(f + s), steps);
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

cudaError_t launch_build(const float *f, uint64_t *W, uint32_t nx, uint32_t ny, uint32_t nz, Workspace &ws,
                         cudaStream_t st)
{
    const uint64_t n = (uint64_t)nx * ny * nz;
    const bool vec = (nx % 4 == 0) && ((uintptr_t)f % 16 == 0) && ((uintptr_t)W % 16 == 0);
    const uint32_t nxq = vec ? nx / 4 : nx;
    const uint32_t nthreads = nxq * ny * nz;
    cudaError_t e;
    {
        PhaseScope ps(kInit, st);
        if (vec)
            k_init<4><<<grid_for(nthreads, 256), 256, 0, st>>>(f, W, nx, ny, nz, nxq, nthreads, ws.status);
        else
            k_init<1><<<grid_for(nthreads, 256), 256, 0, st>>>(f, W, nx, ny, nz, nxq, nthreads, ws.status);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        // descent rounds: at most ~log_{hops}(n) + 2 of them
        PhaseScope ps(kDescend, st);
        for (int round = 0; round < 40; round++) {
            if ((e = cudaMemsetAsync(ws.more, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
            k_descend<<<grid_for(n, 256), 256, 0, st>>>(W, n, 64, ws.more, ws.status);
            count_launch();
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            uint32_t more = 0;
            if ((e = cudaMemcpyAsync(&more, ws.more, sizeof(uint32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                return e;
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
            if (!more) break;
        }
    }
    {
        PhaseScope ps(kMerge, st);
        k_merge<<<grid_for(n, 256), 256, 0, st>>>(W, f, nx, ny, nz, n, ws.status);
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
