// Host-side declarations shared between the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gb300bfs.h"

namespace gb {

// Device status word: the first error a kernel records wins; nothing traps.
struct DevStatus {
    int code;         // 0 or a gb_status
    int where;        // kernel-specific site id
    long long detail; // e.g. the offending index
};

// Per-device library context: the device status word and device limits.
struct Context {
    int device = -1;
    int num_sms = 0;
    DevStatus *status = nullptr;  // device memory
    int bfs_blocks = 0;           // cooperative grid of the BFS kernel (3 blocks per SM)
    int bfs_blocks2 = 0;          // the same with 2 blocks per SM
    int ms_blocks = 0;            // cooperative grid of the multi-source kernel
};

// Context of the current device (created on first use).  Returns nullptr and
// sets the thread's error on failure.
Context *context();

// Thread-local error message.
void set_error(const std::string &msg);
const std::string &last_error();

// Map a CUDA error to a status, recording `what`.
gb_status cuda_fail(cudaError_t e, const char *what);

#define GB_CUDA(call)                                          \
    do {                                                       \
        cudaError_t e__ = (call);                              \
        if (e__ != cudaSuccess) return ::gb::cuda_fail(e__, #call); \
    } while (0)

// Count of kernels this library has launched (process-wide).
void note_launch(unsigned long long n = 1);
unsigned long long launches();

// Process-wide BFS options.
gb_bfs_options &options();
uint64_t timeout_ns();

// Device memory of the library.  Every allocation and free goes through
// these: they count the blocks the library holds (gb_debug_live_allocations)
// and fail on request like an exhausted device (gb_debug_fail_allocations),
// so that tests can check the error paths for leaks without a real failure.
cudaError_t dmalloc_raw(void **p, size_t bytes);
cudaError_t dmalloc_async_raw(void **p, size_t bytes, cudaStream_t s);
cudaError_t dfree(void *p);
cudaError_t dfree_async(void *p, cudaStream_t s);
template <typename T>
inline cudaError_t dmalloc(T **p, size_t bytes)
{
    return dmalloc_raw(reinterpret_cast<void **>(p), bytes);
}
template <typename T>
inline cudaError_t dmalloc_async(T **p, size_t bytes, cudaStream_t s)
{
    return dmalloc_async_raw(reinterpret_cast<void **>(p), bytes, s);
}

// Stream-ordered temporaries.
template <typename T>
inline cudaError_t alloc_async(T **p, size_t count, cudaStream_t s)
{
    return dmalloc_async(p, count * sizeof(T) + (count == 0 ? 16 : 0), s);
}

// The stream-ordered temporaries of one call: every block taken with alloc()
// is freed on the call's stream when the guard goes out of scope, whichever
// way the call returns (a failed allocation or CUDA call midway leaks
// nothing); drop() frees one earlier.  Frees are stream-ordered, so kernels
// already queued on the stream finish with the memory first.
class Scratch {
  public:
    explicit Scratch(cudaStream_t s) : s_(s) {}
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
    ~Scratch()
    {
        for (void *p : p_)
            if (p) dfree_async(p, s_);
    }
    template <typename T>
    cudaError_t alloc(T **p, size_t count)
    {
        const cudaError_t e = alloc_async(p, count, s_);
        if (e == cudaSuccess) p_.push_back(*p);
        return e;
    }
    cudaError_t drop(const void *q)
    {
        for (void *&p : p_)
            if (p == q) {
                void *x = p;
                p = nullptr;
                return dfree_async(x, s_);
            }
        return cudaSuccess;
    }

  private:
    cudaStream_t s_;
    std::vector<void *> p_;
};

// ---------------------------------------------------------------------------
// Radix sort (sort.cu): ascending LSD sort of uint64 keys by bits
// [begin_bit, end_bit), optionally carrying uint32 values.  keys/keys_alt
// (and vals/vals_alt) are two caller buffers of n entries; *keys_out and
// *vals_out receive whichever buffer holds the result.  hist, if given,
// holds the digit counts of every pass of sort_plan(begin_bit, end_bit),
// already counted by the caller; otherwise the sort counts them.
// ---------------------------------------------------------------------------
gb_status radix_sort(uint64_t *keys, uint64_t *keys_alt, uint32_t *vals, uint32_t *vals_alt,
                     int64_t n, int begin_bit, int end_bit, uint64_t **keys_out,
                     uint32_t **vals_out, cudaStream_t s, const unsigned long long *hist = nullptr);
// The sort's passes over bits [begin_bit, end_bit): ceil(bits / 9) passes, the
// first (bits - 8 * passes) of them 9 bits wide and the others 8.  A caller
// that counts the digits itself fills hist[p * RS_RADIX_MAX + digit].
constexpr int RS_MAX_PASSES = 8;
constexpr int RS_MAX_BITS = 9;
constexpr int RS_RADIX_MAX = 1 << RS_MAX_BITS;
struct SortPlan {
    int passes;
    int shift[RS_MAX_PASSES];
    int bits[RS_MAX_PASSES];
};
SortPlan sort_plan(int begin_bit, int end_bit);
// Keys per portion of radix_sort (process-wide; 0 restores the default 2^28).
gb_status set_sort_portion(int64_t keys);
int64_t sort_portion();

// ---------------------------------------------------------------------------
// Graph object.
// ---------------------------------------------------------------------------
}  // namespace gb

struct gb_graph {
    int64_t n = 0;
    int64_t nnz = 0;
    int scale = -1;          // -1 if built from a caller CSR of arbitrary n
    int64_t *off = nullptr;  // device [n+1]
    int32_t *col = nullptr;  // device [nnz]
    uint32_t *nz = nullptr;  // device [ceil(n/32)]: bit v set iff degree(v) >= 1
    int32_t *hub = nullptr;  // device [n]: a neighbour of v of largest degree, or -1
    // device [n]: (hub[v], min(degree(v), 65535)) side by side, one 8-byte load
    // for the bottom-up list walks (65535 means "read the offsets")
    int2 *hd = nullptr;
    int32_t *nzl = nullptr;  // device [nnzv]: the vertices of degree >= 1, ascending
    int64_t nnzv = 0;
    uint32_t *wgt = nullptr; // device [nnz] weights in units of 2^-24 (weighted graphs only)
    uint2 *wadj = nullptr;   // device [nnz] (column, weight) of each row by ascending weight
    // Degree-ordered copy for the batched search (built by build_batched_layout;
    // null until then): vertex i of the copy is rl_perm[i], vertices in order of
    // decreasing degree (ties by id), rows holding their original entry order.
    int64_t *rl_off = nullptr;   // device [n+1]
    int32_t *rl_col = nullptr;   // device [nnz] (padded like col), entries relabelled
    int32_t *rl_perm = nullptr;  // device [n]: copy id -> original id
    int32_t *rl_inv = nullptr;   // device [n]: original id -> copy id
    int device = -1;
};

namespace gb {

// Entries allocated for a graph's columns: nnz rounded up to a multiple of 4
// (at least 4), so that 16-byte loads of an aligned group of four entries
// never leave the allocation.
inline int64_t col_alloc_entries(int64_t nnz) { return nnz < 4 ? 4 : (nnz + 3) & ~int64_t(3); }

// Kernel 1 pieces (csr.cu).
gb_status build_csr(const int64_t *edges, int64_t m, int scale, gb_graph *g, cudaStream_t s);
// Kernel 1 by counting sort (rows scattered, then sorted one by one), m < 2^31 (csr.cu).
gb_status build_csr_counting(const int64_t *edges, int64_t m, int scale, gb_graph *g, cudaStream_t s);
// Generator and kernel 1 fused: the CSR of the Kronecker graph with no edge list (csr.cu).
gb_status kron_csr(int scale, int edgefactor, double a, double b, double c, uint64_t seed_gen,
                   uint64_t seed_perm, gb_graph *g, cudaStream_t s);
// The degree >= 1 bitmap and the hub array of a graph whose CSR is in place (csr.cu).
gb_status build_graph_aux(gb_graph *g, cudaStream_t s);
// The degree-ordered copy of g's CSR for the batched search (csr.cu); a no-op
// if it exists.  Not thread-safe for one graph: the caller serialises.
gb_status build_batched_layout(gb_graph *g, cudaStream_t s);
// The same, serialised with the batched search's own builds (msbfs.cu).
gb_status prepare_batched(gb_graph *g, cudaStream_t s);

// Kernel 1 with the weight row: build_csr, then each entry's least weight (sssp.cu).
gb_status build_csr_weighted(const int64_t *edges, const float *w, int64_t m, int scale, gb_graph *g,
                             cudaStream_t s);

// Kernel 3 (sssp.cu): device statistics of the last search, and the search.
struct SsspDevStats {
    unsigned long long rounds;     // expansion rounds (near queues processed)
    unsigned long long buckets;    // buckets settled
    unsigned long long processed;  // near-queue entries expanded
    unsigned long long scanned;    // edges of the expanded rows
    unsigned long long won;        // relaxations that lowered a distance
    unsigned long long reached;    // vertices with a finite distance
    unsigned long long delta;      // bucket width in units of 2^-24
    unsigned long long phase_ns[4];  // device time: expansion rounds, settle steps, far minima, far splits
};
gb_status sssp_impl(const gb_graph *g, int64_t root, double delta, double *dist, int32_t *parent,
                    SsspDevStats *stats, cudaStream_t s);
gb_status sssp_validate_impl(const gb_graph *g, int64_t root, const int32_t *parent, const double *dist,
                             const int64_t *edges, int64_t m, gb_sssp_validation *out, cudaStream_t s);

// Kronecker generator (gen.cu).
// The weight row of m tuples (gen.cu).
gb_status kron_weights_impl(int64_t m, uint64_t seed_w, float *w, cudaStream_t s);
// The 2m symmetrised kernel-1 keys of the Kronecker tuples, written to keys (gen.cu).
gb_status kron_keys_impl(int scale, int edgefactor, double a, double b, double c,
                         uint64_t seed_gen, uint64_t seed_perm, uint64_t *keys, cudaStream_t s);
gb_status kron_generate_impl(int scale, int edgefactor, double a, double b, double c,
                             uint64_t seed_gen, uint64_t seed_perm, uint64_t seed_shuf,
                             int64_t *edges, cudaStream_t s);

// Per-call statistics written by the BFS kernels (device layout).
constexpr int kStatLevels = 32;
struct BfsDevStats {
    unsigned long long nlevels;
    unsigned long long edges_examined;
    unsigned long long vertices_touched;
    unsigned long long reached;
    unsigned long long td_levels;
    unsigned long long bu_levels;
    unsigned long long init_ns;
    unsigned long long level_ns[kStatLevels];
    unsigned long long level_frontier[kStatLevels];
    int level_dir[kStatLevels];
};

// Single-source BFS (bfs.cu).
// blocks = cooperative grid size (0: the default full-GPU grid); ws = a
// workspace of bfs_workspace_bytes(g) bytes owned by the caller, or nullptr
// to take one from the stream-ordered pool.
// Device validation of one search and its TEPS numerator (validate.cu).
gb_status validate_impl(const gb_graph *g, int64_t root, const int32_t *parent, const int32_t *level,
                        const int64_t *edges, int64_t m, gb_validation *out, cudaStream_t s);
gb_status bfs_impl(const gb_graph *g, int64_t root, int32_t *parent, int32_t *level,
                   BfsDevStats *stats, cudaStream_t s, int blocks = 0, unsigned char *ws = nullptr);
size_t bfs_workspace_bytes(const gb_graph *g);
int bfs_pick_blocks(int num_sms, int minb);

// Multi-source BFS over one graph or a batch of graphs (msbfs.cu).
gb_status msbfs_impl(const gb_graph *g, const int64_t *roots, int k, int32_t *parents,
                     int32_t *levels, BfsDevStats *stats, cudaStream_t s);
gb_status multigraph_impl(const gb_graph *const *gs, int ng, const int64_t *roots, int r,
                          int32_t *const *parents, int32_t *const *levels,
                          BfsDevStats *stats, cudaStream_t s);
int msbfs_pick_blocks(int num_sms);

// Serving (msbfs.cu): one multi-source search state per resident graph, run
// one level per launch with up to 64 queries as bits.
struct MsCtl {
    unsigned long long na;      // active vertices appended for the level
    unsigned long long mf;      // their degree sum
    unsigned long long big;     // (count << 32) | chunks of the big ones
    unsigned long long anynew;  // OR of the bits that reached new vertices
};
struct MsSlots {              // per-bit outputs and start levels
    int32_t *par[64];
    int32_t *lev[64];
    int32_t start[64];
};
struct MsServe;
gb_status ms_serve_create(const gb_graph *g, int blocks, MsServe **out, cudaStream_t s);
void ms_serve_destroy(MsServe *m);
// Device bytes the state holds.
size_t ms_serve_bytes(const MsServe *m);
// Place `count` new queries (bit, root) into the frontier of `level` (the next
// level to run); `table` is the full slot table to upload.
gb_status ms_serve_admit(MsServe *m, int level, int count, const int *bits, const int64_t *roots,
                         const MsSlots *table, cudaStream_t s);
// Run `level` for the bits in `active`; the next level's control record is
// copied to host_ctl (pinned) on the same stream.
gb_status ms_serve_step(MsServe *m, int level, unsigned long long active, MsCtl *host_ctl,
                        cudaStream_t s);

// Last-call statistics bookkeeping (api.cpp).
void note_stats_call(BfsDevStats *dev_stats, cudaStream_t s);
BfsDevStats *stats_buffer();

}  // namespace gb
