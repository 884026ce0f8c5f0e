/*
 * gb300bfs.h -- C ABI of the GB300 Graph500 library (kernels 1, 2 and 3).
 *
 * The library implements the data-parallel part of the Graph500 pipeline that
 * arXiv 2012.13548 ("Graph500 from OCaml-Multicore Perspective") builds on a
 * CPU: Sec. 2.1 (Kronecker edge list), Sec. 2.2 (kernel 1: graph construction
 * as CSR) and Sec. 2.3 (kernel 2: level-synchronous BFS producing a parent and
 * a level array), plus a batched multi-source BFS, a serving loop and Sec. 2.4
 * (kernel 3: single-source shortest paths with parent and distance arrays).
 *
 * Conventions shared by every entry point:
 *   - Every function returns a gb_status; no C++ exception crosses the ABI.
 *     On failure gb_last_error() returns a message (thread-local, valid until
 *     the next call on the same thread).
 *   - "device" pointers are CUDA global-memory pointers of the current device;
 *     "host" pointers are ordinary CPU memory.  The caller owns every array it
 *     passes.  The library owns gb_graph and gb_server objects.
 *   - Work is stream-ordered on the gb_stream given (a cudaStream_t; NULL is
 *     the legacy default stream).  Outputs are valid once that stream has
 *     synchronised.  Calls that must return a size computed on the device
 *     (graph_build_csr) synchronise the stream themselves and say so.
 *   - Errors detected inside a kernel (an edge endpoint out of range, a
 *     bounded device-side wait that ran out) are recorded in a per-device
 *     status word; gb_device_status() synchronises a stream and returns and
 *     clears it.  No kernel traps or asserts.
 *   - Vertex ids are 0-based int64 at the ABI; inside a graph they are stored
 *     as int32 columns, so a graph has at most 2^30 vertices (SCALE <= 30).
 */
#ifndef GB300BFS_H
#define GB300BFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
/* A CUDA stream (cudaStream_t); NULL means the legacy default stream. */
typedef struct CUstream_st *gb_stream;

/* Opaque, library-owned, device-resident CSR graph (Sec. 2.2). */
typedef struct gb_graph gb_graph;

/* Opaque serving loop (resident graphs + admitted queries). */
typedef struct gb_server gb_server;

typedef enum gb_status {
    GB_OK = 0,
    GB_ERR_INVALID = -1,       /* a bad argument (NULL pointer, bad size, bad k) */
    GB_ERR_NOMEM = -2,         /* a device or host allocation failed */
    GB_ERR_CUDA = -3,          /* a CUDA runtime call failed */
    GB_ERR_TIMEOUT = -4,       /* a bounded device-side wait ran out */
    GB_ERR_RANGE = -5,         /* a vertex id outside [0, n) */
    GB_ERR_BUSY = -6,          /* no free slot or memory right now; retry later */
    GB_ERR_UNIMPLEMENTED = -7
} gb_status;

/* Message for the last failure on this thread ("" if none). */
const char *gb_last_error(void);

/* ABI version of this header (incremented on incompatible change). */
int gb_abi_version(void);

/* Number of CUDA kernels this library has launched in this process (all
 * devices, all threads); a caller takes differences to count the kernels of
 * a region.  Library bookkeeping: the paper has no counterpart. */
uint64_t gb_kernel_launches(void);

/* Keys per portion of the device radix sort behind kron_generate and kernel 1
 * (library tuning; the paper has no counterpart).  A sort of more keys than
 * one portion runs portion by portion, each portion's digit counts giving the
 * next portion's output positions; a portion's counts must fit in 30 bits, so
 * 1 <= keys <= 2^28 (the default, and what 0 restores).  Every portion size
 * gives the same result; smaller portions only add kernel launches, and a test
 * uses them to run the chained path, which the default reaches only above
 * 2^28 keys, on small inputs.  Process-wide; applies to later calls.
 * GB_ERR_INVALID outside that range. */
gb_status gb_set_sort_portion(int64_t keys);
int64_t gb_sort_portion(void);

/* Fault injection for tests (library bookkeeping; the paper has no
 * counterpart).  Every device allocation of the library goes through one
 * wrapper; after this call the next `skip` allocations succeed and the `count`
 * after them fail as if the device were out of memory (the call then reports
 * GB_ERR_NOMEM, or, in the server, waits and retries); count = 0 disarms.
 * Process-wide.  gb_debug_live_allocations() is the number of device blocks
 * the library holds at the moment (allocated and not yet freed), so a test
 * can check that a failed call leaks nothing. */
gb_status gb_debug_fail_allocations(int64_t skip, int64_t count);
int64_t gb_debug_live_allocations(void);

/* Synchronise `s`, then return and clear the device status word: GB_OK, or
 * the first GB_ERR_RANGE / GB_ERR_TIMEOUT a kernel recorded since the last
 * call. */
gb_status gb_device_status(gb_stream s);

/* ------------------------------------------------------------------------ */
/* Sec. 2.1: Kronecker edge list.                                            */
/* ------------------------------------------------------------------------ */

/* Generate m = edgefactor * 2^scale edge tuples into `edges` (device,
 * int64 [2][m] structure-of-arrays: row 0 = start vertex, row 1 = end
 * vertex; caller-allocated, 16 * m bytes).  Sec. 2.1: #V = 2^scale,
 * #E = #V * edgefactor; duplicates and self-loops are kept; the vertex
 * numbers are permuted and then the tuples are shuffled.
 * Tuple e draws, for each bit level k < scale, two SplitMix64 values
 * r1, r2 at counters 2(e*scale+k) and 2(e*scale+k)+1 of seed_gen and sets the
 * row/column bits from the quadrant probabilities a, b, c, d = 1-a-b-c
 * (thresholds floor(p * 2^53) against r >> 11).  The permutation ranks
 * vertices by (SplitMix64(seed_perm, v), v); the shuffle puts at position j
 * the tuple of rank j under (SplitMix64(seed_shuf, e), e).
 * Requires 1 <= scale <= 30, edgefactor >= 1, m <= 2^32.  Allocates
 * temporary device memory on `s` (about 24 * m bytes). */
gb_status kron_generate(int scale, int edgefactor, double a, double b, double c,
                        uint64_t seed_gen, uint64_t seed_perm, uint64_t seed_shuf,
                        int64_t *edges, gb_stream s);

/* ------------------------------------------------------------------------ */
/* Sec. 2.2: kernel 1, graph construction (CSR).                             */
/* ------------------------------------------------------------------------ */

/* Build the undirected CSR of `edges` (device int64 [2][m] as produced by
 * kron_generate; read only, may be freed after the call returns) over
 * n = 2^scale vertices.  Row u holds, ascending, every v != u such that
 * (u,v) or (v,u) is a tuple: the graph is symmetrised, self-loops and
 * duplicate edges are dropped (Sec. 2.1 lets the kernels after generation
 * disregard them).  Offsets are int64 [n+1]: an empty row repeats the previous
 * offset and off[n] = nnz (Sec. 2.2).  Columns are int32 [nnz].
 * Synchronises `s` (the column count is needed on the host).  Returns
 * GB_ERR_RANGE if an endpoint is outside [0, 2^scale).  *out receives a
 * library-owned graph; free it with graph_free.  Besides the CSR every graph
 * holds four arrays the search reads: a degree >= 1 bitmap (n/8 bytes), the
 * list of the vertices of degree >= 1 in ascending order (4 bytes each; the
 * first bottom-up level walks it), a hub per vertex (4 * n bytes: a neighbour
 * of largest degree among the first 128 of its row, tested first by the
 * bottom-up step) and, for the bottom-up list walks, each hub again beside
 * the vertex's degree saturated at 65535 (8 * n bytes).  The column array is padded to a multiple of 4
 * entries. */
gb_status graph_build_csr(const int64_t *edges, int64_t m, int scale, gb_graph **out,
                          gb_stream s);

/* Kernel 1 by counting sort instead of a radix sort of the edges (Sec. 2.2
 * builds the CSR from the edges in sorted order; here the rows are counted,
 * the endpoints scattered into them, and each row sorted on its own): the
 * same graph as graph_build_csr, bit for bit, for the same arguments.  Row
 * counts, a scan to row starts, the scatter, per-row sorts by length (a warp
 * up to 32 entries, a block up to 4096, one radix sort of (row, column) keys
 * over the longer rows), the distinct counts scanned into the offsets, and
 * the columns compacted.  Requires m < 2^31; GB_ERR_RANGE otherwise or for an
 * endpoint outside [0, 2^scale).  Synchronises `s`; temporaries about
 * 8 * m + 24 * n bytes plus 16 bytes per entry of the rows longer than 4096. */
gb_status graph_build_csr_counting(const int64_t *edges, int64_t m, int scale, gb_graph **out,
                                   gb_stream s);

/* Sec. 2.1 and Sec. 2.2 fused: the graph graph_build_csr builds from the
 * tuples of kron_generate(scale, edgefactor, a, b, c, seed_gen, seed_perm,
 * any seed_shuf), bit for bit, without the edge list: each generated tuple,
 * relabelled, goes straight into kernel 1's sort as its two symmetric keys.
 * The shuffle of Sec. 2.1 only reorders tuples, which the CSR does not see,
 * so it is skipped (there is no seed_shuf).  The same argument ranges and
 * errors as kron_generate.  Synchronises `s`; temporary device memory about
 * 32 * m bytes (the two separate calls need 16 * m more, for the edge list).
 * *out receives a library-owned graph; free it with graph_free. */
gb_status graph_generate_csr(int scale, int edgefactor, double a, double b, double c,
                             uint64_t seed_gen, uint64_t seed_perm, gb_graph **out,
                             gb_stream s);

/* Wrap a caller-built CSR (device arrays off int64 [n+1], col int32 [nnz]):
 * the arrays are copied into library-owned memory.  The rows must be sorted
 * ascending, free of self-loops and duplicates, and symmetric; only
 * 0 <= col < n and monotone offsets are checked (on the host after a copy).
 * Synchronises `s`. */
gb_status graph_from_csr(const int64_t *off, const int32_t *col, int64_t n, int64_t nnz,
                         gb_graph **out, gb_stream s);

gb_status graph_free(gb_graph *g);

/* Vertex and column counts of g (host outputs). */
gb_status graph_info(const gb_graph *g, int64_t *n, int64_t *nnz);

/* Borrowed device pointers to g's offsets and columns (valid until
 * graph_free). */
gb_status graph_csr_view(const gb_graph *g, const int64_t **off, const int32_t **col);

/* Build g's degree-ordered copy for bfs_batch (a no-op if it exists): the
 * vertices renumbered by decreasing degree (ties by id), each row keeping its
 * entry order, so that the frontier masks of the few vertices holding most of
 * the edge endpoints (Sec. 2.1's skewed degrees) are read from neighbouring
 * lines.  bfs_batch searches a graph that has the copy on it, with the same
 * results (levels, and parents as original ids), and builds it by itself for
 * graphs of 2^25 or more vertices.  It adds 8 (n+1) + 4 nnz + 8 n bytes to the
 * graph until graph_free; GB_ERR_NOMEM leaves the graph as it was.  Part of
 * kernel 1 in the sense of Sec. 4.3 (a structure built once per graph), so
 * not part of the searches' time.  Calls on one graph must not overlap. */
gb_status graph_prepare_batched(gb_graph *g, gb_stream s);

/* ------------------------------------------------------------------------ */
/* Sec. 2.3: kernel 2, breadth-first search.                                 */
/* ------------------------------------------------------------------------ */

/* Options for the BFS entry points (process-wide; applied to later calls).
 *   canonical_parents  0: parent(v) is whichever level-(l-1) neighbour
 *                      claimed v first (any valid Graph500 tree);
 *                      1: parent(v) is the smallest-id neighbour one level
 *                      up (a unique tree, Sec. 2.3.1: the tree follows from
 *                      the level array).  It selects the same for sssp
 *                      (smallest-id neighbour on a shortest path).
 *   alpha, beta        direction switch: top-down -> bottom-up when the
 *                      frontier's edges exceed (unexplored edges)/alpha;
 *                      bottom-up -> top-down when the frontier shrinks below
 *                      n/beta vertices (Beamer et al., SC 2012).
 *   big_degree         frontier vertices of larger degree are split over the
 *                      whole grid in top-down steps.
 *   ms_alpha, ms_beta  the same switch for the multi-source BFS.
 *   timeout_ms         limit of every device-side wait (grid barriers, the
 *                      radix-sort look-back); on expiry the kernel records
 *                      GB_ERR_TIMEOUT and returns.
 *   blocks_per_sm      1, 2 or 3: blocks of the single-source kernel per SM
 *                      (3 trades register spills for more warps; 1 halves the
 *                      grid of 2, which makes the per-level grid barrier
 *                      cheaper on small graphs). */
typedef struct gb_bfs_options {
    int canonical_parents;
    double alpha;
    double beta;
    int big_degree;
    double ms_alpha;
    double ms_beta;
    double timeout_ms;
    int blocks_per_sm;
} gb_bfs_options;

gb_status bfs_get_options(gb_bfs_options *out);
gb_status bfs_set_options(const gb_bfs_options *opt);

/* Single-source BFS from `root` (Sec. 2.3.2, Algorithm "Parallel BFS", run
 * direction-optimised).  parent and level are caller-allocated device int32
 * [n].  On return (after `s` syncs) level[v] is the hop distance from root or
 * -1, parent[root] = root, parent[v] is a neighbour of v with level one less,
 * and parent[v] = -1 for every unreached v.  GB_ERR_RANGE if root is outside
 * [0, n).  One persistent cooperative kernel runs all levels and writes both
 * outputs once, at the end (every entry of parent and level is written);
 * temporary device memory (about 10 * n bytes: bitmaps, the BFS queue, a
 * state byte per vertex and the list of vertices a bottom-up level leaves
 * open) is taken from the stream-ordered pool. */
gb_status bfs(const gb_graph *g, int64_t root, int32_t *parent, int32_t *level, gb_stream s);

/* Multi-source BFS: k (1..64) roots (host array) in one persistent launch,
 * one bit per root in per-vertex masks.  parents and levels are device int32
 * [k][n] (row i belongs to roots[i]); row i equals what bfs() returns for
 * roots[i] (canonical parents in canonical mode, any valid tree otherwise).
 * Roots may repeat. */
gb_status bfs_batch(const gb_graph *g, const int64_t *roots, int k, int32_t *parents,
                    int32_t *levels, gb_stream s);

/* BFS over a batch of ng graphs of different sizes in one launch: r (1..8)
 * roots per graph, roots a host int64 [ng][r] array.  parents[i] and
 * levels[i] (host arrays of ng device pointers) point to int32 [r][n_i]
 * outputs for graph i.  Each result equals the standalone bfs() result. */
gb_status bfs_multi_graph(const gb_graph *const *gs, int ng, const int64_t *roots, int r,
                          int32_t *const *parents, int32_t *const *levels, gb_stream s);

/* Allocation-free single-source BFS (no counterpart in the paper: it exists
 * for callers that may not allocate device memory).  Some callers cannot call
 * cudaMalloc or cudaMallocAsync: a framework whose own allocator has reserved
 * the device's memory, a real-time or embedded host loop that must not stall
 * on the allocator, or code running where allocation is not allowed.  This
 * entry point runs the same kernel as bfs() but keeps every temporary in one
 * file-scope device array built into the library (about 14.4 MB, held on every
 * GPU that loads the library until the process exits), so it never allocates.
 *   off, col   caller's CSR in device memory: off int64 [n+1], col int32
 *              [nnz], rows sorted ascending, symmetric, no self-loops
 *   parent, level  caller's device int32 [n] outputs, as for bfs()
 *   s          the stream it runs on; the call synchronises `s` before it
 *              returns and reports a device-side timeout as GB_ERR_TIMEOUT
 * Limits and rules: n <= 2^20 (1,048,576) vertices, else GB_ERR_RANGE with
 * no work done.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and the grid size; make that first call
 * before any stream capture.  All calls share the one array and it keeps the
 * last call's contents (the header and status word are cleared by each call):
 * calls that overlap on the GPU (other streams, other host threads) race and
 * must not be issued.  Options come from bfs_set_options; bfs_last_stats
 * does not see these calls. */
gb_status bfs_noalloc(const int64_t *off, const int32_t *col, int64_t n, int64_t nnz,
                      int64_t root, int32_t *parent, int32_t *level, gb_stream s);

/* Counters of the last bfs/bfs_batch/bfs_multi_graph call on this thread;
 * synchronises the stream of that call.
 *   nlevels          number of BFS levels (max level + 1)
 *   edges_examined   adjacency entries read (top-down: frontier degrees;
 *                    bottom-up: neighbours tested before the first hit)
 *   vertices_touched frontier vertices expanded plus unvisited vertices
 *                    tested
 *   reached          vertices with level >= 0 (summed over roots)
 *   td_levels, bu_levels  levels run top-down / bottom-up
 *   level_*          per-level device time, frontier and step (see below) */
#define GB_STAT_LEVELS 32
typedef struct gb_bfs_stats {
    int64_t nlevels;
    int64_t edges_examined;
    int64_t vertices_touched;
    int64_t reached;
    int64_t td_levels;
    int64_t bu_levels;
    /* first GB_STAT_LEVELS levels: device time of each level in ns, its
     * frontier size (batched calls: vertices active for any root), and its
     * step (1 top-down, 2 bottom-up) */
    int64_t level_ns[GB_STAT_LEVELS];
    int64_t level_frontier[GB_STAT_LEVELS];
    int32_t level_dir[GB_STAT_LEVELS];
} gb_bfs_stats;

gb_status bfs_last_stats(gb_bfs_stats *out);

/* ------------------------------------------------------------------------ */
/* Sec. 2 outline step 5: validation of a search and its TEPS numerator.     */
/* ------------------------------------------------------------------------ */

/* Verdict of bfs_validate.
 *   code  0 if the output is a valid BFS of g from root, else the first
 *         failing rule of the Graph500 result validation, in the order a
 *         serial check over the vertices, the vertices again and then the
 *         CSR entries meets them:
 *           1  parent(root) != root or level(root) != 0
 *           2  parent(v) = -1 while level(v) != -1, or the reverse
 *           3  a reached v != root whose parent is not a neighbour
 *           4  a reached v != root with level(parent(v)) != level(v) - 1
 *           5  a graph edge with exactly one reached endpoint
 *           6  a graph edge whose endpoint levels differ by more than one
 *           7  root outside [0, n), a parent outside [-1, n) or a level < -1
 *   where  the vertex (rules 1-4, 7) or CSR entry index (5, 6) of that
 *          failure, -1 if code is 0
 *   reached          vertices with level >= 0
 *   component_edges  undirected simple edges among the reached vertices
 *                    (half the CSR entries of their rows)
 *   teps_edges       input tuples whose start vertex is reached, duplicates
 *                    and self-loops included (Sec. 4.3, the Graph500 TEPS
 *                    numerator); -1 when no tuples were given
 *   max_level        largest level, -1 if none */
typedef struct gb_validation {
    int32_t code;
    int32_t max_level;
    int64_t where;
    int64_t reached;
    int64_t component_edges;
    int64_t teps_edges;
} gb_validation;

/* Check parent and level (device int32 [n], as written by bfs or one row of
 * bfs_batch) against g and root on the device, and count the TEPS numerator
 * over edges (device int64 [2][m] input tuples; NULL with m = 0 to skip).
 * Rows of g must be sorted (every graph this library builds is).  Values
 * outside their range are reported as rule 7, never dereferenced.
 * Synchronises s; *out (host) receives the verdict.  Returns GB_OK whenever
 * the check ran, whatever its verdict; GB_ERR_INVALID for NULL arguments or
 * m < 0. */
gb_status bfs_validate(const gb_graph *g, int64_t root, const int32_t *parent,
                       const int32_t *level, const int64_t *edges, int64_t m,
                       gb_validation *out, gb_stream s);

/* ------------------------------------------------------------------------ */
/* Sec. 2.4: kernel 3, single-source shortest paths on the weighted graph.   */
/* ------------------------------------------------------------------------ */

/* The weight row of the 3 x #E tuple matrix (Sec. 2.1): w[j] (device float
 * [m], caller-allocated) = (1 + the top 24 bits of SplitMix64(seed_weight, j))
 * * 2^-24, a multiple of 2^-24 in (0, 1], exact in float.  Weight j belongs
 * to tuple j of the edge list it is used with. */
gb_status kron_weights(int64_t m, uint64_t seed_weight, float *w, gb_stream s);

/* Kernel 1 with weights: the graph graph_build_csr builds from `edges`, and
 * for every CSR entry the least weight among the tuples joining its pair (in
 * either direction; a shortest path uses the lightest copy of an edge).
 * w: device float [m], each in (0, 1]; stored as integer units of 2^-24
 * (rounded to the nearest unit, at least one), so that every path length is
 * an exact sum.  GB_ERR_RANGE for an endpoint outside [0, 2^scale) or a
 * weight outside (0, 1] (NaN included).  Synchronises `s`; the graph also
 * holds 12 * nnz bytes for the weights: one weight per CSR entry and every
 * row again as (column, weight) pairs by ascending weight, which the search
 * reads (built by one radix sort; temporaries about 24 * nnz bytes). */
gb_status graph_build_csr_weighted(const int64_t *edges, const float *w, int64_t m, int scale,
                                   gb_graph **out, gb_stream s);

/* Borrowed device pointer to the weights of a weighted graph (uint32 [nnz],
 * units of 2^-24, parallel to the columns); GB_ERR_INVALID if g has none. */
gb_status graph_weights_view(const gb_graph *g, const uint32_t **wgt);

/* Single-source shortest paths from `root` (Sec. 2.4, Algorithm "Sequential
 * SSSP" computes the same distances; Sec. 4.1 names delta-stepping, which
 * this runs in its near/far form on the device).  g must be built by
 * graph_build_csr_weighted.  delta: bucket width in weight units of 1.0,
 * rounded to a multiple of 2^-24 (at least one unit); <= 0 selects the
 * default 0.0625.  Widths near 0.05-0.1 suit Kronecker graphs with this
 * weight row (a narrower width means more buckets, a wider one more
 * re-expansions within a bucket).  Outputs, caller-allocated device
 * arrays: dist float64 [n] (exact: the least path weight, a multiple of
 * 2^-24; +infinity if unreachable) and parent int32 [n] (parent(root) = root;
 * for a reached v a neighbour u with dist(u) + w(u,v) = dist(v), the
 * smallest-id one when the canonical_parents option is set; -1 if
 * unreachable).  The distances are those of Dijkstra's algorithm exactly; in
 * canonical mode the parent array is the unique canonical tree of them.
 * Allocates about 40 * n bytes of stream-ordered scratch.  GB_ERR_RANGE for
 * a root outside [0, n); GB_ERR_INVALID for an unweighted graph. */
gb_status sssp(const gb_graph *g, int64_t root, double delta, double *dist, int32_t *parent,
               gb_stream s);

/* Statistics of this thread's last sssp call (synchronises its stream).
 *   rounds      expansion rounds (near queues) run
 *   buckets     buckets settled
 *   processed   near-queue entries expanded (a vertex may be expanded
 *               again when its distance drops within its bucket)
 *   scanned     edges of the expanded rows
 *   won         relaxations that lowered a distance
 *   reached     vertices with a finite distance
 *   delta       bucket width used, in weight units of 1.0
 *   phase_ns    device time of the expansion rounds, the settle steps (heavy
 *               edges), the far-list minima and the far-list splits */
typedef struct gb_sssp_stats {
    int64_t rounds;
    int64_t buckets;
    int64_t processed;
    int64_t scanned;
    int64_t won;
    int64_t reached;
    double delta;
    int64_t phase_ns[4];
} gb_sssp_stats;

gb_status sssp_last_stats(gb_sssp_stats *out);

/* Verdict of sssp_validate (the SSSP result rules of the Graph500 benchmark).
 *   code  0 if (parent, dist) is a shortest-path tree of g from root, else
 *         the first failing rule, in the order a serial check meets them
 *         (rule 7 over the vertices, rule 1, rule 2 over the vertices, rules
 *         3-4 over the vertices, rules 5-6 over the CSR entries):
 *           1  parent(root) != root or dist(root) != 0
 *           2  parent(v) = -1 while dist(v) is finite, or the reverse
 *           3  a reached v != root whose parent is not a neighbour
 *           4  a reached v != root with dist(v) != dist(parent) + w(parent, v)
 *           5  a graph edge with exactly one reached endpoint
 *           6  a graph edge (u, v) with dist(v) > dist(u) + w(u, v)
 *           7  root outside [0, n), a parent outside [-1, n), or a distance
 *              that is negative or NaN
 *   where            the vertex (1-4, 7) or CSR entry (5, 6) of the failure
 *   reached          vertices with a finite distance
 *   component_edges  undirected simple edges among them
 *   teps_edges       input tuples whose start vertex is reached (-1 if no
 *                    tuples were given)
 *   max_dist         the largest finite distance */
typedef struct gb_sssp_validation {
    int32_t code;
    int32_t pad;
    int64_t where;
    int64_t reached;
    int64_t component_edges;
    int64_t teps_edges;
    double max_dist;
} gb_sssp_validation;

/* Check (parent, dist) (device arrays as written by sssp) against the
 * weighted graph g on the device; count the TEPS numerator over edges
 * (device int64 [2][m]; NULL with m = 0 to skip).  Synchronises s; returns
 * GB_OK whenever the check ran, whatever its verdict. */
gb_status sssp_validate(const gb_graph *g, int64_t root, const int32_t *parent, const double *dist,
                        const int64_t *edges, int64_t m, gb_sssp_validation *out, gb_stream s);

/* ------------------------------------------------------------------------ */
/* Serving: resident graphs, BFS queries admitted as they arrive.            */
/* ------------------------------------------------------------------------ */

/* How a server serves its graphs (server_default_options fills the defaults).
 *   single_source_min_vertices  graphs with at least this many vertices are
 *                   served by concurrent single-source searches, smaller ones
 *                   as the bits of one multi-source search (default 2^14;
 *                   0 serves every graph by single-source searches)
 *   slots_per_graph concurrent single-source searches per such graph, 1..8
 *                   (default 2), each on its own stream and workspace
 *   full_grid       0 (default): each search of a graph runs on an equal
 *                   share of the SMs, each multi-source graph on a share
 *                   proportional to its size; 1: every launch takes the whole
 *                   grid (the launches then queue behind one another)
 *   verbose         1: print per-graph launch and admission counters to
 *                   stderr when the server is destroyed */
typedef struct gb_server_options {
    int64_t single_source_min_vertices;
    int slots_per_graph;
    int full_grid;
    int verbose;
} gb_server_options;

gb_status server_default_options(gb_server_options *out);

/* Create a server over ng resident graphs (borrowed; they must outlive the
 * server).  Queries are admitted as they arrive, whenever a slot is free and
 * their output buffers (8 * n_graph bytes) fit within mem_budget bytes of
 * device memory; admitted queries run concurrently on the device.  The
 * budget also holds the server's own state (every single-source slot's search
 * workspace, each multi-source search state), counted at creation:
 * GB_ERR_NOMEM if that alone exceeds it.  On a graph of 2^14 or more vertices
 * a slot is one of two concurrent single-source searches, each on its own
 * stream and half of the SMs; on a smaller graph up to 64 queries run
 * together as the bits of one multi-source BFS, a query joining at the next
 * level boundary.  The server runs its own host thread.  Results follow the
 * canonical_parents option like bfs().  server_create uses the default
 * options. */
gb_status server_create(const gb_graph *const *gs, int ng, size_t mem_budget, gb_server **out);
gb_status server_create_with_options(const gb_graph *const *gs, int ng, size_t mem_budget,
                                     const gb_server_options *opt, gb_server **out);

/* Queue a query (graph index, root).  *ticket identifies it.  Never blocks;
 * GB_ERR_RANGE for a bad graph or root. */
gb_status server_submit(gb_server *srv, int graph_id, int64_t root, int64_t *ticket);

/* Poll a query.  Returns GB_OK with *parent/*level set to borrowed device
 * pointers (int32 [n_graph]) once it is done, GB_ERR_BUSY while it is
 * queued or running.  The buffers stay valid until server_release. */
gb_status server_poll(gb_server *srv, int64_t ticket, const int32_t **parent,
                      const int32_t **level);

/* Return a finished query's buffers to the server. */
gb_status server_release(gb_server *srv, int64_t ticket);

/* Cancel a query: a queued one never runs; a running one runs out and its
 * buffers return to the server as soon as it finishes; a finished one is
 * released.  Polling a cancelled ticket gives GB_ERR_INVALID.  GB_ERR_INVALID
 * for an unknown, released or already cancelled ticket. */
gb_status server_cancel(gb_server *srv, int64_t ticket);

/* Counters of a server (host output): its memory budget, the bytes of its own
 * state, the bytes counted against the budget now (that state plus the
 * buffers of admitted queries), and how many queries are queued, running,
 * done (not yet released), released and cancelled. */
typedef struct gb_server_stats {
    int64_t budget_bytes;
    int64_t fixed_bytes;
    int64_t used_bytes;
    int64_t queued;
    int64_t running;
    int64_t done;
    int64_t released;
    int64_t cancelled;
} gb_server_stats;

gb_status server_stats(gb_server *srv, gb_server_stats *out);

/* Replay an open-loop arrival trace: query i arrives t_arrival_s[i] seconds
 * after the call starts (ascending), on graph graph_id[i] from root[i].
 * Blocks until all are done.  latency_ms[i] receives arrival-to-done time
 * (host array, caller-allocated).  Buffers are released as queries
 * finish unless keep_results is nonzero, in which case the caller polls and
 * releases them. */
gb_status server_run_trace(gb_server *srv, int64_t nq, const double *t_arrival_s,
                           const int32_t *graph_id, const int64_t *root, int keep_results,
                           double *latency_ms);

gb_status server_destroy(gb_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* GB300BFS_H */
