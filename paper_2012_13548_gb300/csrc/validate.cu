// Validation of a search's output on the device (Sec. 2, outline step 5: the
// Graph500 benchmark checks every BFS tree it times), and the TEPS numerator
// of Sec. 4.3.  The rules and their order are those of the Graph500 result
// validation:
//
//   1  parent(root) != root or level(root) != 0
//   2  parent(v) = -1 while level(v) != -1, or the reverse
//   3  a reached v != root whose parent is not one of its neighbours
//   4  a reached v != root with level(parent(v)) != level(v) - 1
//   5  a graph edge with exactly one reached endpoint
//   6  a graph edge whose endpoint levels differ by more than one
//   7  root outside [0, n), a parent outside [-1, n) or a level below -1
//
// A serial checker visits the vertices (rules 7 and 2), then the vertices
// again (3, 4), then the CSR entries in order (5, 6), and reports the first
// failure.  Here each of those passes runs in parallel and keeps the smallest
// (index << 3 | rule) of its failures with an atomic minimum; the passes are
// then read in the serial order, so the verdict, and the vertex or CSR entry
// it names, are those of the serial check.
#include "common.cuh"
#include "internal.h"

namespace gb {
namespace {

constexpr int VAL_THREADS = 256;
constexpr int VAL_TILE = 32 * 64;  // CSR entries per warp tile in the edge pass
constexpr unsigned long long kNone = ~0ull;

struct ValAcc {
    unsigned long long first_a;  // vertex pass: rules 7, 2
    unsigned long long first_b;  // vertex pass: rules 3, 4
    unsigned long long first_c;  // CSR entry pass: rules 5, 6
    unsigned long long reached;
    unsigned long long deg_sum;  // degrees of the reached vertices
    unsigned long long teps;
    int max_level;
    int root_bad;
};

__global__ void val_init_kernel(ValAcc *acc)
{
    acc->first_a = kNone;
    acc->first_b = kNone;
    acc->first_c = kNone;
    acc->reached = 0;
    acc->deg_sum = 0;
    acc->teps = 0;
    acc->max_level = -1;
    acc->root_bad = 0;
}

// Rules 1, 7 (values), 2; reached count, degree sum and depth.
__global__ void __launch_bounds__(VAL_THREADS) val_vertex_kernel(const int64_t *__restrict__ off,
                                                                 int64_t n, int64_t root,
                                                                 const int32_t *__restrict__ parent,
                                                                 const int32_t *__restrict__ level,
                                                                 ValAcc *acc)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long reached = 0, deg = 0, first = kNone;
    int maxl = -1;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int32_t p = parent[v], lv = level[v];
        if (v == root && (p != root || lv != 0)) acc->root_bad = 1;
        unsigned code = 0;
        if (p < -1 || (int64_t)p >= n || lv < -1) code = 7;
        else if ((p == -1) != (lv == -1)) code = 2;
        if (code && first == kNone) first = ((unsigned long long)v << 3) | code;
        if (lv >= 0) {
            ++reached;
            deg += (unsigned long long)(off[v + 1] - off[v]);
            maxl = lv > maxl ? lv : maxl;
        }
    }
    // each thread's first failure is its smallest: fold the warp, then one atomic
    for (int o = 16; o >= 1; o >>= 1) {
        const unsigned long long f = __shfl_xor_sync(kFull, first, o);
        first = f < first ? f : first;
        const int m = __shfl_xor_sync(kFull, maxl, o);
        maxl = m > maxl ? m : maxl;
    }
    reached = warp_sum(reached);
    deg = warp_sum(deg);
    if ((threadIdx.x & 31) == 0) {
        if (first != kNone) atomicMin(&acc->first_a, first);
        if (reached) atomicAdd(&acc->reached, reached);
        if (deg) atomicAdd(&acc->deg_sum, deg);
        if (maxl >= 0) atomicMax(&acc->max_level, maxl);
    }
}

// Rules 3, 4.  Rows are sorted, so the parent is looked up by bisection.
// Parents outside [0, n) are the vertex pass's failures and are skipped here.
__global__ void __launch_bounds__(VAL_THREADS) val_parent_kernel(const int64_t *__restrict__ off,
                                                                 const int32_t *__restrict__ col,
                                                                 int64_t n, int64_t root,
                                                                 const int32_t *__restrict__ parent,
                                                                 const int32_t *__restrict__ level,
                                                                 ValAcc *acc)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long first = kNone;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n && first == kNone;
         v += stride) {
        const int32_t lv = level[v];
        const int32_t p = parent[v];
        if (v == root || lv < 0 || p < 0 || (int64_t)p >= n) continue;
        int64_t lo = off[v], hi = off[v + 1];  // search [lo, hi)
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (col[mid] < p) lo = mid + 1;
            else hi = mid;
        }
        unsigned code = 0;
        if (lo >= off[v + 1] || col[lo] != p) code = 3;
        else if (level[p] != lv - 1) code = 4;
        if (code) first = ((unsigned long long)v << 3) | code;
    }
    for (int o = 16; o >= 1; o >>= 1) {
        const unsigned long long f = __shfl_xor_sync(kFull, first, o);
        first = f < first ? f : first;
    }
    if ((threadIdx.x & 31) == 0 && first != kNone) atomicMin(&acc->first_b, first);
}

// Rules 5, 6 over every CSR entry (u, col[e]).  A warp takes a tile of
// VAL_TILE consecutive entries, lane i the entries e0 + i + 32 k; a lane finds
// the row of its first entry by bisection over the offsets and then follows
// the rows forward.
__global__ void __launch_bounds__(VAL_THREADS) val_edge_kernel(const int64_t *__restrict__ off,
                                                               const int32_t *__restrict__ col,
                                                               int64_t n, int64_t nnz,
                                                               const int32_t *__restrict__ level,
                                                               ValAcc *acc)
{
    const unsigned lane = threadIdx.x & 31u;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long first = kNone;
    for (int64_t e0 = gwarp * VAL_TILE; e0 < nnz; e0 += nwarps * VAL_TILE) {
        int64_t e = e0 + lane;
        if (e >= nnz) continue;
        // largest u with off[u] <= e (off[0] = 0 <= e < off[n] = nnz)
        int64_t lo = 0, hi = n;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (off[mid] <= e) lo = mid;
            else hi = mid;
        }
        int64_t u = lo;
        int32_t lu = level[u];
        const int64_t e_end = e0 + VAL_TILE < nnz ? e0 + VAL_TILE : nnz;
        for (; e < e_end && first == kNone; e += 32) {
            int steps = 0;
            while (off[u + 1] <= e && steps < 8) {
                ++u;
                ++steps;
            }
            if (off[u + 1] <= e) {  // a long run of short or empty rows: bisect again
                int64_t a = u, b = n;
                while (b - a > 1) {
                    const int64_t mid = (a + b) >> 1;
                    if (off[mid] <= e) a = mid;
                    else b = mid;
                }
                u = a;
            }
            if (steps) lu = level[u];
            const int32_t v = col[e];
            if (v < 0 || (int64_t)v >= n) continue;  // a CSR built by this library holds none
            const int32_t lw = level[v];
            unsigned code = 0;
            if ((lu < 0) != (lw < 0)) code = 5;
            else if (lu >= 0 && (lu - lw > 1 || lw - lu > 1)) code = 6;
            if (code) first = ((unsigned long long)e << 3) | code;
        }
    }
    for (int o = 16; o >= 1; o >>= 1) {
        const unsigned long long f = __shfl_xor_sync(kFull, first, o);
        first = f < first ? f : first;
    }
    if (lane == 0 && first != kNone) atomicMin(&acc->first_c, first);
}

// TEPS numerator (Sec. 4.3): input tuples whose start vertex was reached,
// duplicates and self-loops included.  Row 0 of the [2][m] tuple array holds
// the start vertices.
__global__ void __launch_bounds__(VAL_THREADS) val_teps_kernel(const int64_t *__restrict__ start,
                                                               int64_t m, int64_t n,
                                                               const int32_t *__restrict__ level,
                                                               ValAcc *acc)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long cnt = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int64_t u = start[e];
        if (u >= 0 && u < n && level[u] >= 0) ++cnt;
    }
    cnt = warp_sum(cnt);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&acc->teps, cnt);
}

}  // namespace

gb_status validate_impl(const gb_graph *g, int64_t root, const int32_t *parent, const int32_t *level,
                        const int64_t *edges, int64_t m, gb_validation *out, cudaStream_t s)
{
    Context *ctx = context();
    if (!ctx) return GB_ERR_CUDA;
    gb_validation r;
    r.code = 0;
    r.where = -1;
    r.reached = 0;
    r.component_edges = 0;
    r.teps_edges = edges ? 0 : -1;
    r.max_level = -1;
    if (root < 0 || root >= g->n) {  // rule 7, checked before anything is read
        r.code = 7;
        r.where = root;
        *out = r;
        return GB_OK;
    }
    ValAcc *acc = nullptr;
    Scratch tmp(s);
    GB_CUDA(tmp.alloc(&acc, 1));
    const int grid = ctx->num_sms * 8;
    val_init_kernel<<<1, 1, 0, s>>>(acc);
    note_launch();
    val_vertex_kernel<<<grid, VAL_THREADS, 0, s>>>(g->off, g->n, root, parent, level, acc);
    note_launch();
    val_parent_kernel<<<grid, VAL_THREADS, 0, s>>>(g->off, g->col, g->n, root, parent, level, acc);
    note_launch();
    if (g->nnz > 0) {
        val_edge_kernel<<<grid, VAL_THREADS, 0, s>>>(g->off, g->col, g->n, g->nnz, level, acc);
        note_launch();
    }
    if (edges && m > 0) {
        val_teps_kernel<<<grid, VAL_THREADS, 0, s>>>(edges, m, g->n, level, acc);
        note_launch();
    }
    GB_CUDA(cudaGetLastError());
    ValAcc h;
    GB_CUDA(cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
    GB_CUDA(tmp.drop(acc));
    GB_CUDA(cudaStreamSynchronize(s));
    r.reached = (int64_t)h.reached;
    r.component_edges = (int64_t)(h.deg_sum / 2);
    if (edges) r.teps_edges = (int64_t)h.teps;
    r.max_level = h.max_level;
    // the serial order: rule 1, the vertex pass, the parent pass, the CSR pass
    const unsigned long long firsts[3] = {h.first_a, h.first_b, h.first_c};
    if (h.root_bad) {
        r.code = 1;
        r.where = root;
    } else {
        for (unsigned long long f : firsts) {
            if (f != kNone) {
                r.code = (int32_t)(f & 7ull);
                r.where = (int64_t)(f >> 3);
                break;
            }
        }
    }
    *out = r;
    return GB_OK;
}

}  // namespace gb
