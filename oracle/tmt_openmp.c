/*
 * CPU baseline (not the oracle): the triplet merge tree computed by the
 * paper's parallel algorithm on the host cores with OpenMP, the counterpart
 * of the OpenMP runs of TMT-SYCL that Table 1 of the paper compares its GPU
 * runs with.
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY. The benchmark times it beside the
 * oracle; the tests check its output against the oracle. The CUDA library
 * never calls, links or includes it, and it shares no code with it or with
 * mt_oracle.c.
 *
 * Algorithm 1 as the paper prints it, with the readings its pseudocode needs:
 *   init    T[u] = (u, u) for every vertex;
 *   merge   every edge (a, b), with S the later end in the order (value,
 *           index), runs Merge(S, a, b) (Algorithm 3): climb a and b along
 *           links whose saddle is at or below S (a root stops a climb), stop
 *           if they meet, else link the later one under the earlier at S with
 *           a 64-bit compare-and-swap (Algorithm 2) and re-insert the link it
 *           held (none if it was a root); a failed compare-and-swap climbs
 *           again;
 *   repair  every vertex u with triplet (s, v): T[u] = (s, Representative(v,
 *           s)) (Algorithms 4 and 5), the representative being the vertex
 *           where the walk along links with saddle at or below s stops.
 * Triplets are packed as (s << 32) | v, as everywhere in this project.
 *
 * Status codes as mt_oracle.c: 0 ok, -1 invalid, -2 too large, -3 non-finite,
 * -6 out of memory, -7 a bounded loop hit its limit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define TMT_OK 0
#define TMT_INVALID (-1)
#define TMT_TOO_LARGE (-2)
#define TMT_NONFINITE (-3)
#define TMT_LIMIT (-7)

#define STEP_LIMIT (1u << 26)

static inline int earlier(const float *f, uint64_t a, uint64_t b)
{
    return f[a] < f[b] || (f[a] == f[b] && a < b);
}

static inline uint64_t ld(const uint64_t *p) { return __atomic_load_n(p, __ATOMIC_RELAXED); }
static inline void st(uint64_t *p, uint64_t v) { __atomic_store_n(p, v, __ATOMIC_RELAXED); }
static inline uint64_t pk(uint64_t s, uint64_t v) { return (s << 32) | v; }
static inline uint64_t hs(uint64_t w) { return w >> 32; }
static inline uint64_t lv(uint64_t w) { return w & 0xFFFFFFFFull; }

/* climb from x through links whose saddle is at or below S; *w gets the
 * word of the vertex where the walk stops */
static uint64_t climb(uint64_t *W, const float *f, uint64_t x, uint64_t S, uint64_t *w, uint32_t *steps)
{
    uint64_t T = ld(W + x);
    for (;;) {
        const uint64_t s = hs(T), t = lv(T);
        if (s == x && t == x) break;
        if (s != S && !earlier(f, s, S)) break;
        x = t;
        T = ld(W + x);
        if (++*steps > STEP_LIMIT) break;
    }
    *w = T;
    return x;
}

static int merge(uint64_t *W, const float *f, uint64_t S, uint64_t a, uint64_t b)
{
    uint64_t u = a, v = b;
    uint32_t steps = 0;
    for (;;) {
        uint64_t Tu, Tv;
        u = climb(W, f, u, S, &Tu, &steps);
        v = climb(W, f, v, S, &Tv, &steps);
        if (++steps > STEP_LIMIT) return 0;
        if (u == v) return 1;
        if (earlier(f, v, u)) {
            uint64_t x = u;
            u = v, v = x;
            x = Tu, Tu = Tv, Tv = x;
        }
        uint64_t expect = Tv;
        if (__atomic_compare_exchange_n(W + v, &expect, pk(S, u), 0, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) {
            if (hs(Tv) == v && lv(Tv) == v) return 1; /* displaced a root */
            S = hs(Tv);                               /* re-insert the displaced link */
            v = lv(Tv);
        }
    }
}

int tmt_openmp(const float *f, uint32_t nx, uint32_t ny, uint32_t nz, int threads, uint64_t *W)
{
    if (!f || !W || nx == 0 || ny == 0 || nz == 0) return TMT_INVALID;
    const uint64_t nxy = (uint64_t)nx * ny, n = nxy * nz;
    if (n >= 0xFFFFFFFFull) return TMT_TOO_LARGE;
    int bad = 0, limit = 0;
    if (threads < 1) threads = 1;
#pragma omp parallel for num_threads(threads) schedule(static) reduction(| : bad)
    for (int64_t u = 0; u < (int64_t)n; u++) {
        bad |= !isfinite(f[u]);
        W[u] = pk((uint64_t)u, (uint64_t)u);
    }
    if (bad) return TMT_NONFINITE;
#pragma omp parallel for num_threads(threads) schedule(dynamic, 4096) reduction(| : limit)
    for (int64_t e = 0; e < (int64_t)(3 * n); e++) {
        const uint64_t u = (uint64_t)e / 3, d = (uint64_t)e % 3;
        const uint64_t x = u % nx, y = (u / nx) % ny, z = u / nxy;
        uint64_t w;
        if (d == 0) {
            if (x + 1 >= nx) continue;
            w = u + 1;
        } else if (d == 1) {
            if (y + 1 >= ny) continue;
            w = u + nx;
        } else {
            if (z + 1 >= nz) continue;
            w = u + nxy;
        }
        const uint64_t S = earlier(f, u, w) ? w : u;
        limit |= !merge(W, f, S, u, w);
    }
    if (limit) return TMT_LIMIT;
#pragma omp parallel for num_threads(threads) schedule(dynamic, 4096) reduction(| : limit)
    for (int64_t i = 0; i < (int64_t)n; i++) {
        const uint64_t u = (uint64_t)i;
        const uint64_t T = ld(W + u), s = hs(T), v = lv(T);
        if (s == u && v == u) continue;
        uint64_t x = v, Tx = ld(W + x);
        uint32_t steps = 0;
        for (;;) {
            const uint64_t sx = hs(Tx), tx = lv(Tx);
            if (sx == x && tx == x) break;
            if (sx != s && !earlier(f, sx, s)) break;
            x = tx;
            Tx = ld(W + x);
            if (++steps > STEP_LIMIT) {
                limit = 1;
                break;
            }
        }
        if (x != v) st(W + u, pk(s, x));
    }
    return limit ? TMT_LIMIT : TMT_OK;
}
