/*
 * libmt -- triplet merge trees of scalar fields on regular grids, on one
 * NVIDIA GB300 (sm_103a).
 *
 * The method is the triplet merge tree of Smirnov and Morozov as adapted to
 * GPUs in "Fast Merge Tree Computation via SYCL" (Nigmetov, Morozov,
 * arXiv 2301.10838): Section 2.1 defines the merge tree, the triplet
 * representation and the algorithms (Algorithms 1-5); Section 3.2 packs the
 * pair (s, v) of each triplet into one 64-bit word so that a single-word
 * compare-and-swap updates it.
 *
 * Conventions shared by every call
 *   grid      nx * ny * nz vertices, x fastest: vertex (x, y, z) has linear
 *             index u = x + nx * (y + ny * z); arrays are C order [nz][ny][nx].
 *             1 <= n = nx*ny*nz < 2^32 - 1 (vertex ids are 32-bit, Section 3.2).
 *   edges     6-neighbourhood: (x+-1, y, z), (x, y+-1, z), (x, y, z+-1).
 *   order     a < b  <=>  f[a] < f[b]  or  (f[a] == f[b] and a < b), IEEE
 *             comparison (-0 == +0). The paper assumes distinct values
 *             (Section 2.1); the linear index breaks ties.
 *   triplet   W[u] = ((uint64_t)s << 32) | v encodes the triplet (u, s, v) of
 *             Section 2.1 in the 64-bit packing of Section 3.2:
 *               s == v == u   u is the deepest vertex of its grid (root);
 *               s == u != v   u lies inside a branch; v is the deepest vertex
 *                             of u's component of the sublevel set at f(u);
 *               s != u        u is a minimum whose branch merges at saddle s
 *                             into the branch of v, v the deepest vertex of
 *                             the component at level f(s).
 *             The result is normalised and minimal (Section 2.1), hence unique:
 *             it does not depend on launch shapes, timing or call mode.
 *   memory    every pointer named d_* is device memory owned by the caller;
 *             h_* is host memory. libmt never frees caller memory and keeps
 *             no pointer after a call returns (the server below owns its own).
 *   streams   `stream` is a cudaStream_t (NULL = the legacy default stream).
 *             Calls enqueue work on it and return without waiting unless
 *             the description says they synchronise.
 *   errors    argument errors are returned at once and enqueue nothing.
 *             Errors found on the device (a non-finite value, a bounded loop
 *             that hit its limit, a full output buffer) are recorded in a
 *             status word inside the workspace and returned by the next call
 *             that synchronises (mt_persistence_pairs, mt_sync_status).
 *             A call that finds the status word already set does no work.
 */
#ifndef MT_H
#define MT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    uint32_t nx, ny, nz;
} mt_grid;

typedef int32_t mt_status;
#define MT_OK 0
#define MT_ERR_INVALID (-1)   /* null pointer, zero side, misaligned or short buffer; caller triplets with ids >= n */
#define MT_ERR_TOO_LARGE (-2) /* n >= 2^32 - 1 */
#define MT_ERR_NONFINITE (-3) /* the field holds NaN or +-inf */
#define MT_ERR_CAPACITY (-4)  /* an output buffer was too small; true count reported */
#define MT_ERR_CUDA (-5)      /* a CUDA runtime call failed */
#define MT_ERR_NOMEM (-6)     /* a device allocation failed (server only) */
#define MT_ERR_TIMEOUT (-7)   /* a bounded device loop hit its iteration limit */
#define MT_ERR_BUSY (-8)      /* server: the ticket is not finished yet */

/* Human-readable name of a status code (static storage). */
const char *mt_status_str(mt_status st);

/* Bytes of device workspace that mt_build_triplets, mt_persistence_pairs and
 * mt_components_at need for grid g (0 if g is invalid). The workspace must be
 * 256-byte aligned and may be reused from call to call on the same stream.
 * Its first 256 bytes hold the status word: zero them once before the first
 * use (mt_build_triplets clears them itself, and so does mt_sync_status);
 * the rest needs no initialisation. */
size_t mt_workspace_bytes(mt_grid g);

/*
 * Triplet merge tree of the sublevel sets of f (Section 2.1, Algorithm 1).
 *   d_f   float32[n], the field, C order [nz][ny][nx]; read only.
 *   d_W   uint64[n], output triplets (layout above); 8-byte aligned.
 *   d_ws  workspace of at least mt_workspace_bytes(g) bytes.
 * Steps, all on the device: validate the values and seed every vertex with
 * its lowest lower neighbour (the initialisation loop of Algorithm 1, seeded
 * along steepest descent), merge every remaining grid edge with 64-bit
 * compare-and-swap (Algorithms 2 and 3), and restore minimality by following
 * representatives (Algorithms 4 and 5). Asynchronous; device-side errors
 * (MT_ERR_NONFINITE, MT_ERR_TIMEOUT) land in the workspace status word.
 */
mt_status mt_build_triplets(const float *d_f, mt_grid g, uint64_t *d_W, void *d_ws, size_t ws_bytes, void *stream);

/* Flags of the _ex calls. MT_SUPERLEVEL: work on the superlevel sets of f,
 * i.e. build the merge tree of -f (the "split tree" of Section 4's setup,
 * the tree the paper's experiments report): minima of -f are maxima of f, and
 * the order is (-f[a], a). mt_components_at_ex with the flag labels the
 * components of {u : f[u] >= t}. The result equals the plain call on -f. */
#define MT_SUPERLEVEL 1u

mt_status mt_build_triplets_ex(const float *d_f, mt_grid g, uint64_t *d_W, void *d_ws, size_t ws_bytes, uint32_t flags,
                               void *stream);

/* mt_build_triplets_ex with a launch configuration cfg (MT_CFG_FOUR_ROUNDS,
 * MT_CFG_REPAIR_256, MT_CFG_LARGE_TILES; MT_CFG_SMALL_TILES is for batches
 * and gives MT_ERR_INVALID, as does any other bit). The triplets do not
 * depend on cfg. */
mt_status mt_build_triplets_cfg(const float *d_f, mt_grid g, uint64_t *d_W, void *d_ws, size_t ws_bytes, uint32_t flags,
                                uint32_t cfg, void *stream);

/* Autotuner for single fields: builds the tree of d_f once per
 * configuration (cfg 0, 2, 4, 6, 8, 10, 12, 14: the single-field knobs) to
 * warm up and three times timed (CUDA events on `stream`), writes the best
 * times to ms[0..7] (in that order; ms holds 8 floats) and the fastest
 * configuration to *best. d_W receives the triplets. Synchronises. */
mt_status mt_build_autotune(const float *d_f, mt_grid g, uint64_t *d_W, void *d_ws, size_t ws_bytes, uint32_t flags,
                            void *stream, float *ms, uint32_t *best);

/*
 * 0-dimensional persistence pairs of the tree in d_W (Section 1: one point
 * (f(a), f(b)) per branch, a a minimum and b the saddle where it merges).
 *   d_pairs   uint32[cap][2]: (minimum u, saddle s) for every u with
 *             W[u].s != u, by ascending u.
 *   h_npairs  host; receives the true number of pairs.
 *   h_root    host; receives the root vertex (W[u] = (u, u)); may be NULL.
 * Synchronises `stream`. Returns the workspace status word if it is set,
 * else MT_ERR_CAPACITY (first cap pairs written, true count in *h_npairs)
 * if the pairs do not fit, else MT_OK. The number of pairs is the number of
 * local minima minus one.
 */
mt_status mt_persistence_pairs(const float *d_f, const uint64_t *d_W, mt_grid g, uint32_t *d_pairs, uint64_t cap,
                               uint64_t *h_npairs, uint32_t *h_root, void *d_ws, size_t ws_bytes, void *stream);

/*
 * Connected components of the sublevel set G_t = {u : f[u] <= t}
 * (Section 2.1), read off the tree: d_labels[u] is the representative of u
 * at level t (Algorithm 4 with the value test f(s) <= t), i.e. the deepest
 * vertex of u's component, or 0xFFFFFFFF when f[u] > t. Asynchronous.
 *   d_labels  uint32[n], output.  t must not be NaN.
 * d_W is followed from vertex to vertex: an id >= n in it sets the status
 * word to MT_ERR_INVALID, and a chain longer than n (a cycle, impossible in
 * a tree) to MT_ERR_TIMEOUT; neither reads outside the arrays.
 */
mt_status mt_components_at(const float *d_f, const uint64_t *d_W, mt_grid g, float t, uint32_t *d_labels,
                           void *d_ws, size_t ws_bytes, void *stream);

mt_status mt_components_at_ex(const float *d_f, const uint64_t *d_W, mt_grid g, float t, uint32_t flags,
                              uint32_t *d_labels, void *d_ws, size_t ws_bytes, void *stream);

/*
 * Persistence simplification (Section 1: the diagram measures the importance
 * of branches, and short branches are noise). A branch -- minimum u, saddle s
 * with W[u].s == s != u -- has persistence p = f(s) - f(u), computed in
 * float32 on the values the order uses (-f with MT_SUPERLEVEL). Simplifying by
 * eps fills every branch of persistence below eps up to its saddle, which
 * removes exactly those pairs from the diagram and leaves all others.
 *
 * mt_simplified_pairs: the pairs (u, s) with p >= eps, by ascending u, with
 * the arguments, synchronisation and return codes of mt_persistence_pairs
 * (eps <= 0 gives all pairs). flags must be those of the build (0 or
 * MT_SUPERLEVEL). eps must not be NaN.
 *
 * mt_simplified_components_at: the components of G_t of the simplified field.
 * A component of G_t whose representative r heads a branch with p < eps lies
 * inside a filled pit and leaves G_t: its vertices get 0xFFFFFFFF. Every other
 * vertex gets the label mt_components_at_ex gives it (the elder rule makes a
 * branch at least as persistent as any branch that merges into it, so no long
 * branch lies inside a filled pit). eps <= 0 gives mt_components_at_ex's
 * labels. Asynchronous; errors as mt_components_at. t and eps must not be NaN.
 */
mt_status mt_simplified_pairs(const float *d_f, const uint64_t *d_W, mt_grid g, float eps, uint32_t flags,
                              uint32_t *d_pairs, uint64_t cap, uint64_t *h_npairs, uint32_t *h_root, void *d_ws,
                              size_t ws_bytes, void *stream);

mt_status mt_simplified_components_at(const float *d_f, const uint64_t *d_W, mt_grid g, float t, float eps,
                                      uint32_t flags, uint32_t *d_labels, void *d_ws, size_t ws_bytes, void *stream);

/*
 * One build that also labels the components of G_t: the triplets of
 * mt_build_triplets_cfg(d_f, g, d_W, d_ws, ws_bytes, flags, cfg, stream) and
 * the labels of mt_simplified_components_at(d_f, d_W, g, t, eps, flags,
 * d_labels, ...) (eps <= 0: those of mt_components_at_ex), bit for bit. The
 * labels are read off the tree inside the repair pass (Algorithm 4 with the
 * value test f(s) <= t, continued from where Algorithm 5 leaves each walk),
 * which saves the separate labelling pass over the field and the triplets.
 *   d_labels  uint32[n], 4-byte aligned, output.  t and eps must not be NaN.
 * Arguments, flags, cfg and errors otherwise as mt_build_triplets_cfg.
 * Asynchronous.
 */
mt_status mt_build_components(const float *d_f, mt_grid g, uint64_t *d_W, float t, float eps, uint32_t flags,
                              uint32_t cfg, uint32_t *d_labels, void *d_ws, size_t ws_bytes, void *stream);

/*
 * The whole path in one call: the triplets and labels of mt_build_components
 * and the pairs of mt_simplified_pairs(d_f, d_W, g, eps, flags, ...) (eps <=
 * 0: those of mt_persistence_pairs), bit for bit, the pairs taken by the
 * same ordered compaction. Arguments as mt_build_components plus the pair
 * outputs of mt_persistence_pairs (d_pairs uint32[cap][2], h_npairs and
 * h_root on the host; h_root may be NULL). Synchronises `stream`; returns
 * the workspace status word if it is set, else MT_ERR_CAPACITY (first cap
 * pairs written, true count in *h_npairs) if the pairs do not fit, else
 * MT_OK.
 */
mt_status mt_build_step(const float *d_f, mt_grid g, uint64_t *d_W, float t, float eps, uint32_t flags, uint32_t cfg,
                        uint32_t *d_labels, uint32_t *d_pairs, uint64_t cap, uint64_t *h_npairs, uint32_t *h_root,
                        void *d_ws, size_t ws_bytes, void *stream);

/*
 * Branch decomposition (Section 2.1: every vertex lies on one branch of the
 * tree; the CPU implementation of Section 3.1 keeps each branch's vertices in
 * a list beside its triplets). A minimum u (W[u].s != u, or the root) heads
 * its own branch; an inner vertex u (W[u] = (u, v), v != u) lies on the
 * branch of v, the deepest vertex of its component at level f(u).
 *   d_order    uint32[n], output: every vertex once, grouped by branch --
 *              branches by ascending id of their minimum -- and each group in
 *              the vertex order (value, then index; the order of -f with
 *              MT_SUPERLEVEL), so that each group starts with its minimum.
 *   d_offsets  uint32[offsets_cap], output: offsets[i] is where group i
 *              starts in d_order, offsets[nbranches] = n.
 *   h_nbranches  host; receives the number of branches (= number of minima).
 *   d_ws       workspace of mt_branches_workspace_bytes(g) bytes (about
 *              21 bytes per vertex), 256-byte aligned.
 * Synchronises `stream`. MT_ERR_CAPACITY (true count in *h_nbranches, order
 * complete, offsets cut off) if offsets_cap < nbranches + 1; MT_ERR_INVALID
 * if d_W holds an id >= n. flags: 0 or MT_SUPERLEVEL, as for the build.
 */
size_t mt_branches_workspace_bytes(mt_grid g);
mt_status mt_branch_decomposition(const float *d_f, const uint64_t *d_W, mt_grid g, uint32_t flags, uint32_t *d_order,
                                  uint32_t *d_offsets, uint64_t offsets_cap, uint64_t *h_nbranches, void *d_ws,
                                  size_t ws_bytes, void *stream);

/*
 * Synchronise `stream` and return (then clear) the workspace status word:
 * MT_OK, MT_ERR_NONFINITE, MT_ERR_TIMEOUT or MT_ERR_CAPACITY.
 */
mt_status mt_sync_status(void *d_ws, void *stream);

/* ------------------------------------------------------------- batches
 * Many fields of uneven sizes in one pass (not in the paper: a batched mode
 * built on the same kernels). Field i occupies elements [off_i, off_i + n_i)
 * of the field arena and of the triplet arena, off_i = n_0 + ... + n_{i-1};
 * its pairs go to pair slots [off_i, off_i + n_i) of the pair arena
 * (uint32[sum n][2]), so every field has room for all its pairs. Vertex ids in
 * triplets and pairs are local to their field. d_npairs[i] receives field
 * i's number of pairs. The results equal those of the single-field calls on
 * each field.
 */
typedef struct {
    uint32_t nfields;
    uint32_t tiles[2];      /* tiles of the two tile shapes */
    uint64_t chunks;        /* pair-compaction chunks */
    uint64_t vertices;      /* sum of n_i */
    uint64_t ws_bytes;      /* workspace the plan needs */
} mt_batch_plan;

/* Workspace for a batch (0 if any grid is invalid); 256-byte aligned. */
size_t mt_batch_workspace_bytes(const mt_grid *h_grids, uint32_t nfields);

/* Validates the grids, writes the field table (arena pointers, offsets,
 * tilings) into the workspace and fills *plan. Synchronises `stream`. Call it
 * again whenever the arenas or the grids change. */
mt_status mt_batch_prepare(const float *d_arena, const mt_grid *h_grids, uint32_t nfields, uint64_t *d_W_arena,
                           uint32_t *d_pairs_arena, void *d_ws, size_t ws_bytes, mt_batch_plan *plan, void *stream);

/* Launch configurations (bits of cfg; 0 is the default). Every
 * configuration gives the same results; they differ only in speed:
 *   MT_CFG_SMALL_TILES  16x16x8 tiles of 256 threads instead of 16x16x16 tiles
 *                       of 512 threads (batches only: small fields leave
 *                       most of a large tile empty)
 *   MT_CFG_FOUR_ROUNDS  4 level buckets per tile instead of 8: the in-tile
 *                       edges are merged, and their vertices repaired, in 4
 *                       rounds by level instead of 8 (Algorithm 1 merges the
 *                       edges in any order)
 *   MT_CFG_REPAIR_256   the repair kernel (Algorithm 5) in CTAs of 256
 *                       threads instead of 512
 *   MT_CFG_LARGE_TILES  32x16x16 tiles of 1024 threads, two CTAs per SM,
 *                       instead of 16x16x16 tiles of 512 threads, four per SM
 *                       (single fields only: fewer edges between tiles
 *                       against fewer warps per SM to issue while a tile
 *                       waits at a round barrier)
 * A batch takes the configurations 0 .. MT_CFG_COUNT - 1; a single field the
 * even ones of 0 .. 15 (MT_CFG_SINGLE_MASK). */
#define MT_CFG_SMALL_TILES 1u
#define MT_CFG_FOUR_ROUNDS 2u
#define MT_CFG_REPAIR_256 4u
#define MT_CFG_LARGE_TILES 8u
#define MT_CFG_COUNT 8
#define MT_CFG_SINGLE_MASK (MT_CFG_FOUR_ROUNDS | MT_CFG_REPAIR_256 | MT_CFG_LARGE_TILES)

/* Enqueues the batched build and pair compaction on `stream`: memsets and
 * kernel launches only, nothing synchronises, so it may be captured in a
 * CUDA graph. cfg is a launch configuration (MT_CFG_* bits, 0 to 7). Device
 * errors land in the workspace status word (mt_sync_status). */
mt_status mt_batch_launch(const mt_batch_plan *plan, int cfg, uint64_t *d_npairs, void *d_ws, size_t ws_bytes,
                          void *stream);

/* mt_batch_prepare followed by mt_batch_launch with variant 0. */
mt_status mt_batch_build(const float *d_arena, const mt_grid *h_grids, uint32_t nfields, uint64_t *d_W_arena,
                         uint32_t *d_pairs_arena, uint64_t *d_npairs, void *d_ws, size_t ws_bytes, void *stream);

/* Autotuner: runs every launch configuration (cfg 0 to MT_CFG_COUNT - 1) of
 * the batch once to warm up and three times timed (CUDA events on
 * `stream`), writes the best time of each to ms[0..MT_CFG_COUNT-1] and the
 * fastest configuration to *best. Synchronises. */
mt_status mt_batch_autotune(const mt_batch_plan *plan, uint64_t *d_npairs, void *d_ws, size_t ws_bytes, void *stream,
                            float *ms, int *best);

/* ------------------------------------------------------------- serving
 * A request loop on one GPU (not in the paper). The server owns a device
 * allocation of hbm_budget_bytes and max_slots CUDA streams. A worker thread
 * admits submitted requests, in arrival order but skipping those that do not
 * fit yet, as soon as a slot and enough of the budget are free, so requests
 * that arrive while others run are started as resources free up and overlap
 * with them on the device. Each request computes the triplet tree of its
 * field, its persistence pairs and its labels at threshold t, exactly as the
 * single-field calls do; the results do not depend on the other requests.
 * A request needs about 20 bytes of the budget per vertex.
 * Fairness: a request that has been overtaken by 8 later requests while it
 * waited for room stops admission behind it until it fits, so a large
 * request is not starved by a stream of small ones.
 */
typedef struct mt_server mt_server;

typedef struct {
    mt_status status;  /* MT_OK, or the request's error */
    uint64_t npairs;   /* number of pairs (also when it exceeded pair_cap) */
    uint32_t root;     /* root vertex */
    uint32_t reused;   /* 1: served from a resident tree (no build), else 0 */
    double t_submit;   /* host steady-clock seconds: submission, */
    double t_admit;    /* admission to a slot, */
    double t_done;     /* results in host memory */
} mt_result;

/* NULL on failure (budget below 1 MiB, max_slots outside 1..64, or the
 * device allocation failed). */
mt_server *mt_server_create(size_t hbm_budget_bytes, int max_slots, int device);

/* Queues a request; *ticket identifies it. h_f (float32[n]) is read and
 * h_pairs (uint32[pair_cap][2], may be NULL) and h_labels (uint32[n], may be
 * NULL) are written by the server until the request completes: keep them
 * alive and untouched until then. Pinned host buffers keep the copies
 * asynchronous; pageable ones work but make the worker wait on each copy.
 * MT_ERR_NOMEM if the request can never fit the budget. */
mt_status mt_server_submit(mt_server *srv, const float *h_f, mt_grid g, float t, uint32_t *h_pairs,
                           uint64_t pair_cap, uint32_t *h_labels, uint64_t *ticket);

/* Resident fields. A request submitted with a nonzero key keeps its field,
 * its triplet tree and its pairs on the device after it completes (about 16
 * bytes of the budget per vertex), under that key. A later request with the
 * same key reuses them: it computes only the labels at its own threshold and
 * copies the stored pairs, and its result has reused = 1; h_f may then be
 * NULL. A key names one field: a request whose grid differs from the resident
 * one's fails with MT_ERR_INVALID, and a field passed under a key that is
 * already resident is not read. A request for a key whose build is still
 * running waits for it. Resident entries that no running request uses are
 * evicted, least recently used first, when an admission needs their memory;
 * a request with h_f == NULL whose key is no longer resident fails with
 * MT_ERR_INVALID. The results equal those of a one-off request. */
mt_status mt_server_submit_resident(mt_server *srv, uint64_t key, const float *h_f, mt_grid g, float t,
                                    uint32_t *h_pairs, uint64_t pair_cap, uint32_t *h_labels, uint64_t *ticket);

/* Drops the resident entry of key as soon as no request uses it.
 * MT_ERR_INVALID if the key is not resident. */
mt_status mt_server_evict(mt_server *srv, uint64_t key);

/* Number of resident entries that are built, and the device bytes they hold. */
mt_status mt_server_resident(mt_server *srv, uint64_t *count, uint64_t *bytes);

/* Non-blocking: MT_OK and *r once the request is done (the result is then
 * forgotten), MT_ERR_BUSY while it is pending or running. */
mt_status mt_server_poll(mt_server *srv, uint64_t ticket, mt_result *r);

/* Blocks until the request is done, then as mt_server_poll. */
mt_status mt_server_wait(mt_server *srv, uint64_t ticket, mt_result *r);

/* Finishes queued and running requests, then frees the server. */
void mt_server_destroy(mt_server *srv);

/* ------------------------------------------------------------- wide ids
 * Grids of 2^32 vertices and more (Section 3.2 caps ids at 32 bits because
 * SYCL has no double-word compare-and-swap; Section 5 names wider ids as
 * future work). Each triplet is one 128-bit word of two 64-bit ids,
 *   W[2u] = s, W[2u + 1] = v      (uint64[n][2], 16-byte aligned),
 * with the meaning of the 64-bit packing above; it is updated with a 128-bit
 * compare-and-swap. Ids have 34 bits: 1 <= n < 2^34 (every grid whose field
 * and triplets fit in one GPU's memory); larger grids get MT_ERR_TOO_LARGE.
 * The results are those of the 32-bit calls with the ids widened, for any n.
 * The build runs the tile kernel of mt_build_triplets (16-bit ids inside a
 * tile), merges the edges between tiles with the 128-bit compare-and-swap and
 * repairs: about 3x slower per vertex than the 32-bit calls.
 *   flags      0 or MT_SUPERLEVEL, as for mt_build_triplets_ex.
 *   d_ws       mt_wide_workspace_bytes(g) bytes, 256-byte aligned; status
 *              word as for the other calls (mt_sync_status reads it).
 * mt_build_triplets_wide is asynchronous. mt_persistence_pairs_wide writes
 * (minimum u, saddle s) rows of uint64[cap][2] by ascending u, synchronises
 * and returns like mt_persistence_pairs (root in *h_root). mt_components_at_wide
 * writes uint64[n] labels (0xFFFFFFFFFFFFFFFF outside G_t), asynchronously.
 */
size_t mt_wide_workspace_bytes(mt_grid g);
mt_status mt_build_triplets_wide(const float *d_f, mt_grid g, uint64_t *d_W, void *d_ws, size_t ws_bytes,
                                 uint32_t flags, void *stream);
mt_status mt_persistence_pairs_wide(const uint64_t *d_W, mt_grid g, uint64_t *d_pairs, uint64_t cap,
                                    uint64_t *h_npairs, uint64_t *h_root, void *d_ws, size_t ws_bytes, void *stream);
mt_status mt_components_at_wide(const float *d_f, const uint64_t *d_W, mt_grid g, float t, uint32_t flags,
                                uint64_t *d_labels, void *d_ws, size_t ws_bytes, void *stream);

/*
 * Persistence pairs for callers that cannot allocate device memory. The paper
 * has no counterpart to this call; it exists because some callers may not
 * obtain a workspace: a host application may own all device memory through
 * its own pool and forbid further cudaMalloc, or a latency-critical path may
 * not take the synchronisation and latency of an allocation. It computes the
 * same pairs, root and count as mt_persistence_pairs (same arguments minus
 * the workspace) and synchronises `stream` in the same way.
 *   Scratch: one array of about 1 MiB compiled into libmt. It exists on every
 *            GPU that loads the library and stays allocated there until the
 *            process exits. This call allocates and frees nothing.
 *   Limit:   n <= 2^30 vertices (1024^3); larger grids get MT_ERR_TOO_LARGE
 *            before anything is enqueued.
 *   Set-up:  every call looks up the array's device address
 *            (cudaGetSymbolAddress) in the context current on the calling
 *            thread, so the address always belongs to that context, primary
 *            or not. The first call on a device may also load libmt's device
 *            code there: make that first call before any stream capture
 *            begins.
 *   Sharing: every call uses the same array, which keeps the last call's
 *            contents (each call clears what must start at zero). Calls that
 *            overlap on the GPU (other streams, other host threads) race on it
 *            and must be serialised by the caller.
 *   Status:  device errors recorded by mt_build_triplets live in that call's
 *            workspace and are not reported here.
 */
mt_status mt_persistence_pairs_noalloc(const float *d_f, const uint64_t *d_W, mt_grid g, uint32_t *d_pairs,
                                       uint64_t cap, uint64_t *h_npairs, uint32_t *h_root, void *stream);

/* ------------------------------------------------------------- tracing
 * Not part of the paper's method: diagnostics for benchmarks and profiling.
 * When enabled, every step (tile, merge, repair, pairs, labels, branches)
 * is bracketed by CUDA events on the stream it runs on; mt_trace_read waits
 * for the recorded events and returns the accumulated device time per step.
 */
typedef struct {
    char name[16];
    unsigned long long calls;
    double total_ms;
} mt_phase_time;

void mt_trace_enable(int on);
/* Fills up to max_entries rows (steps with at least one call), returns how
 * many steps have data; reset != 0 clears the totals afterwards. */
int mt_trace_read(mt_phase_time *out, int max_entries, int reset);
/* Number of kernels libmt has launched in this process so far. */
unsigned long long mt_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* MT_H */
