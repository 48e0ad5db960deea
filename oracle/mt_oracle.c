/*
 * CPU oracle for the triplet merge tree of a scalar field on a 6-connected
 * regular grid.
 *
 * TEST INFRASTRUCTURE ONLY. It exists to check the CUDA library. Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg load it; the
 * library never calls, links or includes anything here, and this file shares
 * no code with it.
 *
 * Everything is plain, sequential and written for a reader to check against
 * the paper by eye; nothing is tuned.
 *
 * Conventions
 *   grid      nx * ny * nz vertices, linear index u = x + nx*(y + ny*z)
 *   edges     the 6-neighbourhood (x+-1, y+-1, z+-1) inside the grid
 *   order     a before b  <=>  f[a] < f[b]  or  (f[a] == f[b] and a < b).
 *             The paper assumes distinct values (Section 2.1 sorts the
 *             vertices, Algorithm 1 tests f(v) < f(u)); ties are broken by the
 *             linear index so that the order is total. IEEE comparison is
 *             used, so -0 and +0 are equal values.
 *   triplet   W[u] = (s << 32) | v encodes the triplet (u, s, v) of
 *             Section 2.1 ("Triplet merge trees"): the branch born at u
 *             merges into the branch of v at s. (u, u, u) marks the global
 *             minimum; (u, u, v) a vertex inside a branch.
 *
 * Status codes: 0 ok, -1 invalid argument, -2 too large (n >= 2^32 - 1),
 *               -3 non-finite value, -4 capacity too small, -6 out of memory.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_INVALID (-1)
#define OR_TOO_LARGE (-2)
#define OR_NONFINITE (-3)
#define OR_CAPACITY (-4)
#define OR_NOMEM (-6)

/* ---------------------------------------------------------------- order */

/* a before b in the total order (value, linear index). */
static int before(const float *f, uint64_t a, uint64_t b)
{
    if (f[a] < f[b]) return 1;
    if (f[a] > f[b]) return 0;
    return a < b;
}

typedef struct {
    float val;
    uint32_t idx;
} keyed_t;

static int cmp_keyed(const void *pa, const void *pb)
{
    const keyed_t *a = (const keyed_t *)pa, *b = (const keyed_t *)pb;
    if (a->val < b->val) return -1;
    if (a->val > b->val) return 1;
    if (a->idx < b->idx) return -1;
    if (a->idx > b->idx) return 1;
    return 0;
}

/* ------------------------------------------------------------ grid helpers */

typedef struct {
    uint64_t nx, ny, nz, n;
} grid_t;

static int make_grid(uint32_t nx, uint32_t ny, uint32_t nz, grid_t *g)
{
    if (nx == 0 || ny == 0 || nz == 0) return OR_INVALID;
    g->nx = nx;
    g->ny = ny;
    g->nz = nz;
    g->n = (uint64_t)nx * ny * nz;
    if (g->n >= 0xFFFFFFFFull) return OR_TOO_LARGE;
    return OR_OK;
}

/* Writes the in-grid 6-neighbours of u into nb[], returns how many. */
static int neighbours(const grid_t *g, uint64_t u, uint64_t nb[6])
{
    uint64_t x = u % g->nx, y = (u / g->nx) % g->ny, z = u / (g->nx * g->ny);
    int k = 0;
    if (x > 0) nb[k++] = u - 1;
    if (x + 1 < g->nx) nb[k++] = u + 1;
    if (y > 0) nb[k++] = u - g->nx;
    if (y + 1 < g->ny) nb[k++] = u + g->nx;
    if (z > 0) nb[k++] = u - g->nx * g->ny;
    if (z + 1 < g->nz) nb[k++] = u + g->nx * g->ny;
    return k;
}

static int check_finite(const float *f, uint64_t n)
{
    for (uint64_t i = 0; i < n; i++)
        if (!isfinite(f[i])) return OR_NONFINITE;
    return OR_OK;
}

static uint64_t pack(uint64_t s, uint64_t v) { return (s << 32) | v; }

/* ------------------------------------------------------------ union-find */

static uint32_t uf_find(uint32_t *parent, uint32_t x)
{
    while (parent[x] != x) {
        parent[x] = parent[parent[x]]; /* path halving */
        x = parent[x];
    }
    return x;
}

/* --------------------------------------------------------- merge tree */

/*
 * The serial merge-tree construction of Section 2.1 ("Merge Trees"): sort the
 * vertices, sweep them in order and use union-find to decide whether the
 * current vertex starts a component (a minimum), joins one, or merges several.
 * The triplets are read off the sweep:
 *   - no swept neighbour: u is a minimum and starts a branch, W[u] = (u, u);
 *   - otherwise let e be the swept component whose deepest vertex cmin[e] comes
 *     first in the order (the elder); W[u] = (u, cmin[e]) because cmin[e] is
 *     the deepest vertex of u's component at level f(u) (minimality, 2.1);
 *   - every other swept component r dies at u: the branch born at cmin[r]
 *     merges into cmin[e] at u, W[cmin[r]] = (u, cmin[e]).
 * The result satisfies normalisation and minimality, which make the triplet
 * representation unique (Section 2.1).
 *
 * The sort and the sweep are separate entry points so that a caller can time
 * them separately; oracle_merge_tree runs both.
 */
int oracle_sort_order(const float *f, uint32_t nx, uint32_t ny, uint32_t nz, uint32_t *order)
{
    grid_t g;
    int st = make_grid(nx, ny, nz, &g);
    if (st) return st;
    if (!f || !order) return OR_INVALID;
    st = check_finite(f, g.n);
    if (st) return st;
    keyed_t *k = (keyed_t *)malloc(g.n * sizeof(keyed_t));
    if (!k) return OR_NOMEM;
    for (uint64_t i = 0; i < g.n; i++) {
        k[i].val = f[i];
        k[i].idx = (uint32_t)i;
    }
    qsort(k, g.n, sizeof(keyed_t), cmp_keyed);
    for (uint64_t i = 0; i < g.n; i++) order[i] = k[i].idx;
    free(k);
    return OR_OK;
}

/*
 * The same order written as one 64-bit integer per vertex, so that a library
 * sort of plain integers can stand in for qsort with a comparison function
 * (at 1024^3 vertices qsort takes minutes). Unsigned comparison of two keys
 * gives the order (value, linear index):
 *   high 32 bits  the value's bit pattern made monotone in the value: -0 is
 *                 first replaced by +0 (IEEE comparison treats them as equal),
 *                 a non-negative value then gets its sign bit set (so it lies
 *                 above every negative one and grows with its magnitude), and
 *                 a negative value has all its bits flipped (so a larger
 *                 magnitude gives a smaller key);
 *   low 32 bits   the linear index (n < 2^32), which breaks ties.
 * Sorting the keys ascending and keeping their low halves gives the same
 * order as oracle_sort_order.
 */
int oracle_order_keys(const float *f, uint32_t nx, uint32_t ny, uint32_t nz, uint64_t *keys)
{
    grid_t g;
    int st = make_grid(nx, ny, nz, &g);
    if (st) return st;
    if (!f || !keys) return OR_INVALID;
    st = check_finite(f, g.n);
    if (st) return st;
    for (uint64_t i = 0; i < g.n; i++) {
        float x = f[i];
        if (x == 0.0f) x = 0.0f; /* -0 -> +0 */
        uint32_t b;
        memcpy(&b, &x, sizeof b);
        uint32_t m = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
        keys[i] = ((uint64_t)m << 32) | i;
    }
    return OR_OK;
}

int oracle_sweep(const float *f, uint32_t nx, uint32_t ny, uint32_t nz, const uint32_t *order, uint64_t *W)
{
    grid_t g;
    int st = make_grid(nx, ny, nz, &g);
    if (st) return st;
    if (!f || !order || !W) return OR_INVALID;
    uint32_t *parent = (uint32_t *)malloc(g.n * sizeof(uint32_t));
    uint32_t *cmin = (uint32_t *)malloc(g.n * sizeof(uint32_t));
    unsigned char *swept = (unsigned char *)calloc(g.n, 1);
    if (!parent || !cmin || !swept) {
        free(parent);
        free(cmin);
        free(swept);
        return OR_NOMEM;
    }
    for (uint64_t k = 0; k < g.n; k++) {
        uint64_t u = order[k];
        uint64_t nb[6];
        int nn = neighbours(&g, u, nb);
        uint32_t roots[6];
        int nr = 0;
        for (int j = 0; j < nn; j++) {
            if (!swept[nb[j]]) continue;
            uint32_t r = uf_find(parent, (uint32_t)nb[j]);
            int seen = 0;
            for (int q = 0; q < nr; q++)
                if (roots[q] == r) seen = 1;
            if (!seen) roots[nr++] = r;
        }
        if (nr == 0) {
            W[u] = pack(u, u);
            parent[u] = (uint32_t)u;
            cmin[u] = (uint32_t)u;
        } else {
            uint32_t e = roots[0];
            for (int q = 1; q < nr; q++)
                if (before(f, cmin[roots[q]], cmin[e])) e = roots[q];
            W[u] = pack(u, cmin[e]);
            for (int q = 0; q < nr; q++) {
                if (roots[q] == e) continue;
                W[cmin[roots[q]]] = pack(u, cmin[e]);
                parent[roots[q]] = e;
            }
            parent[u] = e;
        }
        swept[u] = 1;
    }
    free(parent);
    free(cmin);
    free(swept);
    return OR_OK;
}

int oracle_merge_tree(const float *f, uint32_t nx, uint32_t ny, uint32_t nz, uint64_t *W)
{
    grid_t g;
    int st = make_grid(nx, ny, nz, &g);
    if (st) return st;
    if (!f || !W) return OR_INVALID;
    uint32_t *order = (uint32_t *)malloc(g.n * sizeof(uint32_t));
    if (!order) return OR_NOMEM;
    st = oracle_sort_order(f, nx, ny, nz, order);
    if (!st) st = oracle_sweep(f, nx, ny, nz, order, W);
    free(order);
    return st;
}

/* ---------------------------------------------------------------- pairs */

/*
 * 0-dimensional persistence pairs (Section 1: one diagram point per branch
 * (a, b), a a minimum and b a saddle): every u with W[u].s != u gives the
 * pair (u, W[u].s), listed by ascending u. Roots are the u with W[u] = (u,u).
 * Writes at most cap pairs; *npairs gets the true count; returns
 * OR_CAPACITY if it exceeded cap.
 */
int oracle_pairs(const uint64_t *W, uint64_t n, uint32_t *pairs, uint64_t cap, uint64_t *npairs,
                 uint64_t *nroots, uint32_t *root)
{
    if (!W || !npairs || !nroots) return OR_INVALID;
    uint64_t k = 0, r = 0;
    for (uint64_t u = 0; u < n; u++) {
        uint64_t s = W[u] >> 32, v = W[u] & 0xFFFFFFFFull;
        if (s != u) {
            if (k < cap && pairs) {
                pairs[2 * k] = (uint32_t)u;
                pairs[2 * k + 1] = (uint32_t)s;
            }
            k++;
        } else if (v == u) {
            if (r == 0 && root) *root = (uint32_t)u;
            r++;
        }
    }
    *npairs = k;
    *nroots = r;
    return k > cap ? OR_CAPACITY : OR_OK;
}

/* ------------------------------------------------------------ components */

/*
 * Connected components of the sublevel set G_t = {u : f[u] <= t}
 * (Section 2.1), built directly from the field with union-find over the
 * grid edges and without any merge tree. label[u] is the deepest vertex of
 * u's component (the first in the total order), or 0xFFFFFFFF if f[u] > t.
 */
int oracle_components(const float *f, uint32_t nx, uint32_t ny, uint32_t nz, float t, uint32_t *label)
{
    grid_t g;
    int st = make_grid(nx, ny, nz, &g);
    if (st) return st;
    if (!f || !label) return OR_INVALID;
    st = check_finite(f, g.n);
    if (st) return st;
    uint32_t *parent = (uint32_t *)malloc(g.n * sizeof(uint32_t));
    uint32_t *deep = (uint32_t *)malloc(g.n * sizeof(uint32_t));
    if (!parent || !deep) {
        free(parent);
        free(deep);
        return OR_NOMEM;
    }
    for (uint64_t u = 0; u < g.n; u++) parent[u] = (uint32_t)u;
    for (uint64_t u = 0; u < g.n; u++) {
        if (!(f[u] <= t)) continue;
        uint64_t nb[6];
        int nn = neighbours(&g, u, nb);
        for (int j = 0; j < nn; j++) {
            if (!(f[nb[j]] <= t)) continue;
            uint32_t a = uf_find(parent, (uint32_t)u), b = uf_find(parent, (uint32_t)nb[j]);
            if (a != b) parent[a] = b;
        }
    }
    for (uint64_t u = 0; u < g.n; u++) deep[u] = 0xFFFFFFFFu;
    for (uint64_t u = 0; u < g.n; u++) {
        if (!(f[u] <= t)) continue;
        uint32_t r = uf_find(parent, (uint32_t)u);
        if (deep[r] == 0xFFFFFFFFu || before(f, u, deep[r])) deep[r] = (uint32_t)u;
    }
    for (uint64_t u = 0; u < g.n; u++)
        label[u] = (f[u] <= t) ? deep[uf_find(parent, (uint32_t)u)] : 0xFFFFFFFFu;
    free(parent);
    free(deep);
    return OR_OK;
}

/* ------------------------------------------------------------ point query */

/* Open-addressing set of vertex ids, used so that one query touches only the
 * vertices it visits (the full-size grids have ~1e9 vertices). */
typedef struct {
    uint64_t *slot;
    uint64_t mask, count;
} idset_t;

static int set_init(idset_t *s, uint64_t budget)
{
    uint64_t cap = 64;
    while (cap < 2 * budget + 2) cap <<= 1;
    s->slot = (uint64_t *)malloc(cap * sizeof(uint64_t));
    if (!s->slot) return OR_NOMEM;
    for (uint64_t i = 0; i < cap; i++) s->slot[i] = UINT64_MAX;
    s->mask = cap - 1;
    s->count = 0;
    return OR_OK;
}

/* returns 1 if inserted, 0 if already present */
static int set_add(idset_t *s, uint64_t key)
{
    uint64_t h = (key * 0x9E3779B97F4A7C15ull) >> 17;
    for (uint64_t i = h & s->mask;; i = (i + 1) & s->mask) {
        if (s->slot[i] == key) return 0;
        if (s->slot[i] == UINT64_MAX) {
            s->slot[i] = key;
            s->count++;
            return 1;
        }
    }
}

static void set_clear(idset_t *s)
{
    for (uint64_t i = 0; i <= s->mask; i++) s->slot[i] = UINT64_MAX;
    s->count = 0;
}

/* Deepest vertex of u's component of {w : w before-or-equal lvl}, by BFS.
 * Returns 1 and *deep on success, 0 if more than budget vertices were seen. */
static int bfs_deepest(const float *f, const grid_t *g, uint64_t u, uint64_t lvl, uint64_t budget,
                       idset_t *seen, uint64_t *queue, uint64_t *deep)
{
    set_clear(seen);
    uint64_t head = 0, tail = 0;
    set_add(seen, u);
    queue[tail++] = u;
    uint64_t best = u;
    while (head < tail) {
        uint64_t x = queue[head++];
        if (before(f, x, best)) best = x;
        uint64_t nb[6];
        int nn = neighbours(g, x, nb);
        for (int j = 0; j < nn; j++) {
            uint64_t w = nb[j];
            if (!(w == lvl || before(f, w, lvl))) continue;
            if (!set_add(seen, w)) continue;
            if (tail >= budget) return 0;
            queue[tail++] = w;
        }
    }
    *deep = best;
    return 1;
}

/* binary min-heap of vertex ids under the total order */
static void heap_push(const float *f, uint64_t *h, uint64_t *len, uint64_t x)
{
    uint64_t i = (*len)++;
    h[i] = x;
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (!before(f, h[i], h[p])) break;
        uint64_t t = h[i];
        h[i] = h[p];
        h[p] = t;
        i = p;
    }
}

static uint64_t heap_pop(const float *f, uint64_t *h, uint64_t *len)
{
    uint64_t top = h[0];
    h[0] = h[--(*len)];
    uint64_t i = 0;
    for (;;) {
        uint64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < *len && before(f, h[l], h[m])) m = l;
        if (r < *len && before(f, h[r], h[m])) m = r;
        if (m == i) break;
        uint64_t t = h[i];
        h[i] = h[m];
        h[m] = t;
        i = m;
    }
    return top;
}

/*
 * The triplet of one vertex u, straight from the definitions of Section 2.1,
 * touching only the vertices near u:
 *   - u has a neighbour before it: u is inside a branch, W[u] = (u, v) with v
 *     the deepest vertex of u's component of G_{f(u)} (breadth-first search);
 *   - otherwise u is a minimum. Flood outwards from u always taking the
 *     earliest vertex on the boundary (priority flood); the first vertex
 *     before u that the flood reaches joins u's component at level s, the
 *     latest vertex taken so far. W[u] = (s, v), v the deepest vertex of u's
 *     component of G_{f(s)}. If the flood covers the grid without meeting a
 *     vertex before u, u is the global minimum and W[u] = (u, u).
 * Returns 1 with *Wu set, 0 if the query would visit more than `budget`
 * vertices, or a negative status.
 */
static int point_triplet(const float *f, grid_t g, uint64_t u, uint64_t budget, uint64_t *s_out, uint64_t *v_out)
{
    if (!f || !s_out || !v_out || u >= g.n || budget < 1) return OR_INVALID;
    if (budget > g.n) budget = g.n;
    idset_t seen;
    if (set_init(&seen, 6 * budget + 8)) return OR_NOMEM;
    uint64_t *buf = (uint64_t *)malloc((6 * budget + 8) * sizeof(uint64_t));
    if (!buf) {
        free(seen.slot);
        return OR_NOMEM;
    }
    int ok = 0;
    uint64_t nb[6];
    int nn = neighbours(&g, u, nb), has_lower = 0;
    for (int j = 0; j < nn; j++)
        if (before(f, nb[j], u)) has_lower = 1;
    if (has_lower) {
        uint64_t deep;
        ok = bfs_deepest(f, &g, u, u, budget, &seen, buf, &deep);
        if (ok) *s_out = u, *v_out = deep;
    } else {
        /* priority flood from the minimum u */
        uint64_t len = 0, level = u, popped = 0;
        int found = 0;
        set_add(&seen, u);
        for (int j = 0; j < nn; j++)
            if (set_add(&seen, nb[j])) heap_push(f, buf, &len, nb[j]);
        while (len > 0) {
            uint64_t x = heap_pop(f, buf, &len);
            if (before(f, x, u)) {
                found = 1;
                break;
            }
            if (before(f, level, x)) level = x;
            if (++popped >= budget) break;
            uint64_t xb[6];
            int xn = neighbours(&g, x, xb);
            for (int j = 0; j < xn; j++)
                if (set_add(&seen, xb[j])) heap_push(f, buf, &len, xb[j]);
        }
        if (found) {
            uint64_t deep;
            ok = bfs_deepest(f, &g, u, level, budget, &seen, buf, &deep);
            if (ok) *s_out = level, *v_out = deep;
        } else if (len == 0 && popped < budget) {
            *s_out = u, *v_out = u; /* flood covered the whole grid */
            ok = 1;
        }
    }
    free(seen.slot);
    free(buf);
    return ok;
}

int oracle_point_triplet(const float *f, uint32_t nx, uint32_t ny, uint32_t nz, uint64_t u, uint64_t budget,
                         uint64_t *Wu)
{
    grid_t g;
    int st = make_grid(nx, ny, nz, &g);
    if (st) return st;
    if (!Wu) return OR_INVALID;
    uint64_t s, v;
    int r = point_triplet(f, g, u, budget, &s, &v);
    if (r == 1) *Wu = pack(s, v);
    return r;
}

/* ------------------------------------------------------------ wide ids */

/*
 * The same constructions with 64-bit vertex ids, for grids of 2^32 vertices
 * and more (Section 3.2 limits the packed pair to 32-bit ids; Section 5
 * names wider ids as future work). Each triplet is two 64-bit words,
 * W2[2u] = s and W2[2u + 1] = v. Only the id width differs from the
 * functions above.
 */
static int make_grid_wide(uint32_t nx, uint32_t ny, uint32_t nz, grid_t *g)
{
    if (nx == 0 || ny == 0 || nz == 0) return OR_INVALID;
    g->nx = nx;
    g->ny = ny;
    g->nz = nz;
    g->n = (uint64_t)nx * ny * nz;
    return OR_OK;
}

typedef struct {
    float val;
    uint64_t idx;
} keyed_wide_t;

static int cmp_keyed_wide(const void *pa, const void *pb)
{
    const keyed_wide_t *a = (const keyed_wide_t *)pa, *b = (const keyed_wide_t *)pb;
    if (a->val < b->val) return -1;
    if (a->val > b->val) return 1;
    if (a->idx < b->idx) return -1;
    if (a->idx > b->idx) return 1;
    return 0;
}

static uint64_t uf_find_wide(uint64_t *parent, uint64_t x)
{
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

/* The sort and sweep of oracle_sort_order / oracle_sweep with 64-bit ids. */
int oracle_merge_tree_wide(const float *f, uint32_t nx, uint32_t ny, uint32_t nz, uint64_t *W2)
{
    grid_t g;
    int st = make_grid_wide(nx, ny, nz, &g);
    if (st) return st;
    if (!f || !W2) return OR_INVALID;
    st = check_finite(f, g.n);
    if (st) return st;
    keyed_wide_t *k = (keyed_wide_t *)malloc(g.n * sizeof(keyed_wide_t));
    uint64_t *parent = (uint64_t *)malloc(g.n * sizeof(uint64_t));
    uint64_t *cmin = (uint64_t *)malloc(g.n * sizeof(uint64_t));
    unsigned char *swept = (unsigned char *)calloc(g.n, 1);
    if (!k || !parent || !cmin || !swept) {
        free(k);
        free(parent);
        free(cmin);
        free(swept);
        return OR_NOMEM;
    }
    for (uint64_t i = 0; i < g.n; i++) {
        k[i].val = f[i];
        k[i].idx = i;
    }
    qsort(k, g.n, sizeof(keyed_wide_t), cmp_keyed_wide);
    for (uint64_t q = 0; q < g.n; q++) {
        uint64_t u = k[q].idx;
        uint64_t nb[6];
        int nn = neighbours(&g, u, nb);
        uint64_t roots[6];
        int nr = 0;
        for (int j = 0; j < nn; j++) {
            if (!swept[nb[j]]) continue;
            uint64_t r = uf_find_wide(parent, nb[j]);
            int seen = 0;
            for (int c = 0; c < nr; c++)
                if (roots[c] == r) seen = 1;
            if (!seen) roots[nr++] = r;
        }
        if (nr == 0) {
            W2[2 * u] = u;
            W2[2 * u + 1] = u;
            parent[u] = u;
            cmin[u] = u;
        } else {
            uint64_t e = roots[0];
            for (int c = 1; c < nr; c++)
                if (before(f, cmin[roots[c]], cmin[e])) e = roots[c];
            W2[2 * u] = u;
            W2[2 * u + 1] = cmin[e];
            for (int c = 0; c < nr; c++) {
                if (roots[c] == e) continue;
                W2[2 * cmin[roots[c]]] = u;
                W2[2 * cmin[roots[c]] + 1] = cmin[e];
                parent[roots[c]] = e;
            }
            parent[u] = e;
        }
        swept[u] = 1;
    }
    free(k);
    free(parent);
    free(cmin);
    free(swept);
    return OR_OK;
}

/* oracle_components with 64-bit labels (all ones outside G_t). */
int oracle_components_wide(const float *f, uint32_t nx, uint32_t ny, uint32_t nz, float t, uint64_t *label)
{
    grid_t g;
    int st = make_grid_wide(nx, ny, nz, &g);
    if (st) return st;
    if (!f || !label) return OR_INVALID;
    st = check_finite(f, g.n);
    if (st) return st;
    uint64_t *parent = (uint64_t *)malloc(g.n * sizeof(uint64_t));
    uint64_t *deep = (uint64_t *)malloc(g.n * sizeof(uint64_t));
    if (!parent || !deep) {
        free(parent);
        free(deep);
        return OR_NOMEM;
    }
    for (uint64_t u = 0; u < g.n; u++) parent[u] = u;
    for (uint64_t u = 0; u < g.n; u++) {
        if (!(f[u] <= t)) continue;
        uint64_t nb[6];
        int nn = neighbours(&g, u, nb);
        for (int j = 0; j < nn; j++) {
            if (!(f[nb[j]] <= t)) continue;
            uint64_t a = uf_find_wide(parent, u), b = uf_find_wide(parent, nb[j]);
            if (a != b) parent[a] = b;
        }
    }
    for (uint64_t u = 0; u < g.n; u++) deep[u] = UINT64_MAX;
    for (uint64_t u = 0; u < g.n; u++) {
        if (!(f[u] <= t)) continue;
        uint64_t r = uf_find_wide(parent, u);
        if (deep[r] == UINT64_MAX || before(f, u, deep[r])) deep[r] = u;
    }
    for (uint64_t u = 0; u < g.n; u++) label[u] = (f[u] <= t) ? deep[uf_find_wide(parent, u)] : UINT64_MAX;
    free(parent);
    free(deep);
    return OR_OK;
}

/* oracle_point_triplet for grids of any size: out[0] = s, out[1] = v. */
int oracle_point_triplet_wide(const float *f, uint32_t nx, uint32_t ny, uint32_t nz, uint64_t u, uint64_t budget,
                              uint64_t *out)
{
    grid_t g;
    int st = make_grid_wide(nx, ny, nz, &g);
    if (st) return st;
    if (!out) return OR_INVALID;
    return point_triplet(f, g, u, budget, out, out + 1);
}
