// C ABI of the library (include/gb300bfs.h): argument checks, error
// reporting, the per-device context and the graph objects.  Every compute
// step runs in the CUDA kernels of gen.cu, sort.cu, csr.cu, bfs.cu, msbfs.cu,
// validate.cu and sssp.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "gb300bfs.h"
#include "internal.h"

namespace gb {

namespace {
std::atomic<unsigned long long> g_launches{0};
std::atomic<long long> g_live_allocs{0};  // device blocks the library holds
std::mutex g_fail_mu;                      // injected allocation failures
long long g_fail_skip = 0, g_fail_count = 0;
thread_local std::string t_err;
std::mutex g_ctx_mu;
std::vector<Context *> g_ctx;  // indexed by device

gb_bfs_options g_opt = {
    0,       // canonical_parents
    14.0,    // alpha
    24.0,    // beta
    256,     // big_degree
    16.0,    // ms_alpha
    32.0,    // ms_beta
    5000.0,  // timeout_ms
    2,       // blocks_per_sm
};

// last-call statistics of this thread
struct StatsSlot {
    int device = -1;
    BfsDevStats *dev = nullptr;
    cudaStream_t stream = nullptr;
    bool valid = false;
};
thread_local StatsSlot t_stats;

// last sssp call of this thread
struct SsspSlot {
    int device = -1;
    SsspDevStats *dev = nullptr;
    cudaStream_t stream = nullptr;
    bool valid = false;
};
thread_local SsspSlot t_sssp;

SsspDevStats *sssp_stats_buffer()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    if (t_sssp.dev && t_sssp.device == dev) return t_sssp.dev;
    if (t_sssp.dev) {
        int old = 0;
        cudaGetDevice(&old);
        cudaSetDevice(t_sssp.device);
        gb::dfree(t_sssp.dev);
        cudaSetDevice(old);
        t_sssp.dev = nullptr;
    }
    if (gb::dmalloc((void **)&t_sssp.dev, sizeof(SsspDevStats)) != cudaSuccess) return nullptr;
    t_sssp.device = dev;
    t_sssp.valid = false;
    return t_sssp.dev;
}

// Free every device array of a graph (any may be null) and the graph.
void destroy_graph(gb_graph *g)
{
    void *arrays[] = {g->off, g->col, g->nz, g->hub, g->nzl, g->hd, g->rl_off, g->rl_col, g->rl_perm, g->rl_inv, g->wgt, g->wadj};
    for (void *p : arrays)
        if (p) gb::dfree(p);
    delete g;
}

gb_status check_graph(const gb_graph *g)
{
    if (!g || !g->off) {
        set_error("NULL or freed graph");
        return GB_ERR_INVALID;
    }
    return GB_OK;
}

}  // namespace

// True if an injected failure takes this allocation.
static bool injected_failure()
{
    std::lock_guard<std::mutex> lk(g_fail_mu);
    if (g_fail_count <= 0) return false;
    if (g_fail_skip > 0) {
        --g_fail_skip;
        return false;
    }
    --g_fail_count;
    return true;
}

cudaError_t dmalloc_raw(void **p, size_t bytes)
{
    if (injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) g_live_allocs.fetch_add(1);
    return e;
}

cudaError_t dmalloc_async_raw(void **p, size_t bytes, cudaStream_t s)
{
    if (injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e == cudaSuccess) g_live_allocs.fetch_add(1);
    return e;
}

cudaError_t dfree(void *p)
{
    if (!p) return cudaSuccess;
    g_live_allocs.fetch_sub(1);
    return cudaFree(p);
}

cudaError_t dfree_async(void *p, cudaStream_t s)
{
    if (!p) return cudaSuccess;
    g_live_allocs.fetch_sub(1);
    return cudaFreeAsync(p, s);
}

void set_error(const std::string &msg) { t_err = msg; }
void note_launch(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long launches() { return g_launches.load(std::memory_order_relaxed); }
const std::string &last_error() { return t_err; }

gb_status cuda_fail(cudaError_t e, const char *what)
{
    t_err = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return GB_ERR_NOMEM;
    return GB_ERR_CUDA;
}

gb_bfs_options &options() { return g_opt; }

uint64_t timeout_ns()
{
    double ms = g_opt.timeout_ms > 0 ? g_opt.timeout_ms : 5000.0;
    return (uint64_t)(ms * 1e6);
}

Context *context()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cuda_fail(e, "cudaGetDevice");
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    if ((int)g_ctx.size() <= dev) g_ctx.resize(dev + 1, nullptr);
    if (g_ctx[dev]) return g_ctx[dev];
    Context *c = new (std::nothrow) Context();
    if (!c) {
        t_err = "out of host memory";
        return nullptr;
    }
    c->device = dev;
    if ((e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev)) !=
            cudaSuccess ||
        (e = gb::dmalloc((void **)&c->status, sizeof(DevStatus))) != cudaSuccess ||
        (e = cudaMemset(c->status, 0, sizeof(DevStatus))) != cudaSuccess) {
        cuda_fail(e, "library context");
        delete c;
        return nullptr;
    }
    // keep freed stream-ordered memory in the pool between calls
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    c->bfs_blocks = bfs_pick_blocks(c->num_sms, 3);
    c->bfs_blocks2 = bfs_pick_blocks(c->num_sms, 2);
    c->ms_blocks = msbfs_pick_blocks(c->num_sms);
    g_ctx[dev] = c;
    return c;
}

BfsDevStats *stats_buffer()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    if (t_stats.dev && t_stats.device == dev) return t_stats.dev;
    if (t_stats.dev) {
        int old = 0;
        cudaGetDevice(&old);
        cudaSetDevice(t_stats.device);
        gb::dfree(t_stats.dev);
        cudaSetDevice(old);
        t_stats.dev = nullptr;
    }
    if (gb::dmalloc((void **)&t_stats.dev, sizeof(BfsDevStats)) != cudaSuccess) return nullptr;
    t_stats.device = dev;
    t_stats.valid = false;
    return t_stats.dev;
}

void note_stats_call(BfsDevStats *dev_stats, cudaStream_t s)
{
    (void)dev_stats;
    t_stats.stream = s;
    t_stats.valid = true;
}

}  // namespace gb

using namespace gb;

namespace {

cudaStream_t as_stream(gb_stream s) { return reinterpret_cast<cudaStream_t>(s); }

// Default bucket width of kernel 3 (weight units of 1.0).
constexpr double kDefaultDelta = 0.0625;

template <typename F>
gb_status guarded(F &&f)
{
    try {
        return f();
    } catch (const std::bad_alloc &) {
        set_error("out of host memory");
        return GB_ERR_NOMEM;
    } catch (...) {
        set_error("internal error");
        return GB_ERR_INVALID;
    }
}

}  // namespace

extern "C" {

const char *gb_last_error(void) { return last_error().c_str(); }

int gb_abi_version(void) { return 1; }

uint64_t gb_kernel_launches(void) { return launches(); }

gb_status gb_set_sort_portion(int64_t keys) { return set_sort_portion(keys); }

gb_status gb_debug_fail_allocations(int64_t skip, int64_t count)
{
    if (skip < 0 || count < 0) {
        set_error("gb_debug_fail_allocations: skip and count must be >= 0");
        return GB_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_fail_mu);
    g_fail_skip = skip;
    g_fail_count = count;
    return GB_OK;
}

int64_t gb_debug_live_allocations(void) { return (int64_t)g_live_allocs.load(); }

int64_t gb_sort_portion(void) { return sort_portion(); }

gb_status gb_device_status(gb_stream s)
{
    return guarded([&]() -> gb_status {
        Context *ctx = context();
        if (!ctx) return GB_ERR_CUDA;
        GB_CUDA(cudaStreamSynchronize(as_stream(s)));
        DevStatus h;
        GB_CUDA(cudaMemcpy(&h, ctx->status, sizeof(h), cudaMemcpyDeviceToHost));
        if (h.code != 0) {
            GB_CUDA(cudaMemset(ctx->status, 0, sizeof(DevStatus)));
            set_error("device status " + std::to_string(h.code) + " at site " +
                      std::to_string(h.where) + " (detail " + std::to_string(h.detail) + ")");
            return (gb_status)h.code;
        }
        return GB_OK;
    });
}

gb_status kron_generate(int scale, int edgefactor, double a, double b, double c, uint64_t seed_gen,
                        uint64_t seed_perm, uint64_t seed_shuf, int64_t *edges, gb_stream s)
{
    return guarded([&]() {
        if (!(a >= 0 && b >= 0 && c >= 0 && a + b + c <= 1.0 + 1e-12)) {
            set_error("kron_generate: initiator probabilities must be >= 0 with a+b+c <= 1");
            return GB_ERR_INVALID;
        }
        return kron_generate_impl(scale, edgefactor, a, b, c, seed_gen, seed_perm, seed_shuf,
                                  edges, as_stream(s));
    });
}

gb_status graph_build_csr(const int64_t *edges, int64_t m, int scale, gb_graph **out, gb_stream s)
{
    return guarded([&]() {
        if (!out || scale < 1 || scale > 30 || m < 0 || (m > 0 && !edges)) {
            set_error("graph_build_csr: need out != NULL, 1 <= scale <= 30, m >= 0");
            return GB_ERR_INVALID;
        }
        *out = nullptr;
        gb_graph *g = new gb_graph();
        gb_status rc = build_csr(edges, m, scale, g, as_stream(s));
        if (rc != GB_OK) {
            destroy_graph(g);
            return rc;
        }
        *out = g;
        return GB_OK;
    });
}

gb_status graph_build_csr_counting(const int64_t *edges, int64_t m, int scale, gb_graph **out,
                                   gb_stream s)
{
    return guarded([&]() {
        if (!out || scale < 1 || scale > 30 || m < 0 || (m > 0 && !edges)) {
            set_error("graph_build_csr_counting: need out != NULL, 1 <= scale <= 30, m >= 0");
            return GB_ERR_INVALID;
        }
        *out = nullptr;
        gb_graph *g = new gb_graph();
        gb_status rc = build_csr_counting(edges, m, scale, g, as_stream(s));
        if (rc != GB_OK) {
            destroy_graph(g);
            return rc;
        }
        *out = g;
        return GB_OK;
    });
}

gb_status kron_weights(int64_t m, uint64_t seed_weight, float *w, gb_stream s)
{
    return guarded([&]() -> gb_status {
        if (m < 0 || (m > 0 && !w)) {
            set_error("kron_weights: need m >= 0 and w != NULL");
            return GB_ERR_INVALID;
        }
        return kron_weights_impl(m, seed_weight, w, as_stream(s));
    });
}

gb_status graph_build_csr_weighted(const int64_t *edges, const float *w, int64_t m, int scale,
                                   gb_graph **out, gb_stream s)
{
    return guarded([&]() {
        if (!out || scale < 1 || scale > 30 || m < 0 || (m > 0 && (!edges || !w))) {
            set_error("graph_build_csr_weighted: need out != NULL, 1 <= scale <= 30, m >= 0, "
                      "edges and w != NULL if m > 0");
            return GB_ERR_INVALID;
        }
        *out = nullptr;
        gb_graph *g = new gb_graph();
        gb_status rc = build_csr_weighted(edges, w, m, scale, g, as_stream(s));
        if (rc != GB_OK) {
            cudaStreamSynchronize(as_stream(s));
            destroy_graph(g);
            return rc;
        }
        *out = g;
        return GB_OK;
    });
}

gb_status graph_weights_view(const gb_graph *g, const uint32_t **wgt)
{
    gb_status rc = check_graph(g);
    if (rc != GB_OK) return rc;
    if (!g->wgt) {
        set_error("graph_weights_view: the graph has no weights");
        return GB_ERR_INVALID;
    }
    if (wgt) *wgt = g->wgt;
    return GB_OK;
}

gb_status sssp(const gb_graph *g, int64_t root, double delta, double *dist, int32_t *parent,
               gb_stream s)
{
    return guarded([&]() -> gb_status {
        gb_status rc = check_graph(g);
        if (rc != GB_OK) return rc;
        if (!dist || !parent || std::isnan(delta)) {
            set_error("sssp: NULL output or NaN delta");
            return GB_ERR_INVALID;
        }
        if (root < 0 || root >= g->n) {
            set_error("sssp: root outside [0, n)");
            return GB_ERR_RANGE;
        }
        SsspDevStats *st = sssp_stats_buffer();
        if (!st) return cuda_fail(cudaErrorMemoryAllocation, "sssp stats buffer");
        rc = sssp_impl(g, root, delta > 0 ? delta : kDefaultDelta, dist, parent, st, as_stream(s));
        if (rc == GB_OK) {
            t_sssp.stream = as_stream(s);
            t_sssp.valid = true;
        }
        return rc;
    });
}

gb_status sssp_last_stats(gb_sssp_stats *out)
{
    return guarded([&]() -> gb_status {
        if (!out) {
            set_error("sssp_last_stats: NULL");
            return GB_ERR_INVALID;
        }
        if (!t_sssp.valid || !t_sssp.dev) {
            set_error("sssp_last_stats: no sssp call on this thread yet");
            return GB_ERR_INVALID;
        }
        SsspDevStats h;
        GB_CUDA(cudaStreamSynchronize(t_sssp.stream));
        GB_CUDA(cudaMemcpy(&h, t_sssp.dev, sizeof(h), cudaMemcpyDeviceToHost));
        out->rounds = (int64_t)h.rounds;
        out->buckets = (int64_t)h.buckets;
        out->processed = (int64_t)h.processed;
        out->scanned = (int64_t)h.scanned;
        out->won = (int64_t)h.won;
        out->reached = (int64_t)h.reached;
        out->delta = (double)h.delta / 16777216.0;
        for (int k = 0; k < 4; ++k) out->phase_ns[k] = (int64_t)h.phase_ns[k];
        return GB_OK;
    });
}

gb_status sssp_validate(const gb_graph *g, int64_t root, const int32_t *parent, const double *dist,
                        const int64_t *edges, int64_t m, gb_sssp_validation *out, gb_stream s)
{
    return guarded([&]() -> gb_status {
        if (!g || !parent || !dist || !out || m < 0 || (m > 0 && !edges)) {
            set_error("sssp_validate: need g, parent, dist, out != NULL, m >= 0, edges != NULL if m > 0");
            return GB_ERR_INVALID;
        }
        gb_status rc = check_graph(g);
        if (rc != GB_OK) return rc;
        return sssp_validate_impl(g, root, parent, dist, m > 0 ? edges : nullptr, m, out, as_stream(s));
    });
}

gb_status graph_generate_csr(int scale, int edgefactor, double a, double b, double c,
                             uint64_t seed_gen, uint64_t seed_perm, gb_graph **out, gb_stream s)
{
    return guarded([&]() {
        if (!out) {
            set_error("graph_generate_csr: out == NULL");
            return GB_ERR_INVALID;
        }
        if (!(a >= 0 && b >= 0 && c >= 0 && a + b + c <= 1.0 + 1e-12)) {
            set_error("graph_generate_csr: initiator probabilities must be >= 0 with a+b+c <= 1");
            return GB_ERR_INVALID;
        }
        *out = nullptr;
        gb_graph *g = new gb_graph();
        gb_status rc = kron_csr(scale, edgefactor, a, b, c, seed_gen, seed_perm, g, as_stream(s));
        if (rc != GB_OK) {
            destroy_graph(g);
            return rc;
        }
        *out = g;
        return GB_OK;
    });
}

gb_status graph_from_csr(const int64_t *off, const int32_t *col, int64_t n, int64_t nnz,
                         gb_graph **out, gb_stream s)
{
    return guarded([&]() -> gb_status {
        if (!out || !off || n < 1 || n > (int64_t(1) << 30) || nnz < 0 || (nnz > 0 && !col)) {
            set_error("graph_from_csr: need out, off != NULL, 1 <= n <= 2^30, nnz >= 0");
            return GB_ERR_INVALID;
        }
        *out = nullptr;
        Context *ctx = context();
        if (!ctx) return GB_ERR_CUDA;
        cudaStream_t st = as_stream(s);
        std::vector<int64_t> hoff(n + 1);
        std::vector<int32_t> hcol(nnz);
        GB_CUDA(cudaMemcpyAsync(hoff.data(), off, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        if (nnz) GB_CUDA(cudaMemcpyAsync(hcol.data(), col, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaStreamSynchronize(st));
        if (hoff[0] != 0 || hoff[n] != nnz) {
            set_error("graph_from_csr: off[0] must be 0 and off[n] must equal nnz");
            return GB_ERR_INVALID;
        }
        for (int64_t i = 0; i < n; ++i)
            if (hoff[i + 1] < hoff[i]) {
                set_error("graph_from_csr: offsets must be non-decreasing");
                return GB_ERR_INVALID;
            }
        for (int64_t j = 0; j < nnz; ++j)
            if (hcol[j] < 0 || hcol[j] >= n) {
                set_error("graph_from_csr: a column is outside [0, n)");
                return GB_ERR_RANGE;
            }
        gb_graph *g = new gb_graph();
        g->n = n;
        g->nnz = nnz;
        g->scale = -1;
        g->device = ctx->device;
        cudaError_t e;
        if ((e = gb::dmalloc(&g->off, (n + 1) * sizeof(int64_t))) != cudaSuccess ||
            (e = gb::dmalloc(&g->col, col_alloc_entries(nnz) * sizeof(int32_t))) != cudaSuccess ||
            (e = cudaMemcpyAsync(g->off, off, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
            (nnz && (e = cudaMemcpyAsync(g->col, col, nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, st)) != cudaSuccess) ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess) {
            gb::dfree(g->off);
            gb::dfree(g->col);
            delete g;
            return cuda_fail(e, "graph_from_csr");
        }
        gb_status rc = build_graph_aux(g, st);
        if (rc == GB_OK && (e = cudaStreamSynchronize(st)) != cudaSuccess) rc = cuda_fail(e, "graph_from_csr");
        if (rc != GB_OK) {
            destroy_graph(g);
            return rc;
        }
        *out = g;
        return GB_OK;
    });
}

gb_status graph_free(gb_graph *g)
{
    return guarded([&]() -> gb_status {
        if (!g) return GB_OK;
        cudaDeviceSynchronize();
        destroy_graph(g);
        return GB_OK;
    });
}

gb_status graph_prepare_batched(gb_graph *g, gb_stream s)
{
    return guarded([&]() -> gb_status {
        gb_status rc = check_graph(g);
        if (rc != GB_OK) return rc;
        return gb::prepare_batched(g, as_stream(s));
    });
}

gb_status graph_info(const gb_graph *g, int64_t *n, int64_t *nnz)
{
    gb_status rc = check_graph(g);
    if (rc != GB_OK) return rc;
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    return GB_OK;
}

gb_status graph_csr_view(const gb_graph *g, const int64_t **off, const int32_t **col)
{
    gb_status rc = check_graph(g);
    if (rc != GB_OK) return rc;
    if (off) *off = g->off;
    if (col) *col = g->col;
    return GB_OK;
}

gb_status bfs_get_options(gb_bfs_options *out)
{
    if (!out) {
        set_error("bfs_get_options: NULL");
        return GB_ERR_INVALID;
    }
    *out = options();
    return GB_OK;
}

gb_status bfs_set_options(const gb_bfs_options *opt)
{
    if (!opt || !(opt->alpha > 0) || !(opt->beta > 0) || opt->big_degree < 1 ||
        !(opt->ms_alpha > 0) || !(opt->ms_beta > 0) || !(opt->timeout_ms > 0) ||
        opt->blocks_per_sm < 1 || opt->blocks_per_sm > 3) {
        set_error("bfs_set_options: alpha, beta, ms_alpha, ms_beta, timeout_ms must be > 0, "
                  "big_degree >= 1 and blocks_per_sm 1, 2 or 3");
        return GB_ERR_INVALID;
    }
    options() = *opt;
    return GB_OK;
}

gb_status bfs(const gb_graph *g, int64_t root, int32_t *parent, int32_t *level, gb_stream s)
{
    return guarded([&]() -> gb_status {
        gb_status rc = check_graph(g);
        if (rc != GB_OK) return rc;
        if (!parent || !level) {
            set_error("bfs: NULL output");
            return GB_ERR_INVALID;
        }
        if (root < 0 || root >= g->n) {
            set_error("bfs: root outside [0, n)");
            return GB_ERR_RANGE;
        }
        BfsDevStats *st = stats_buffer();
        if (!st) return cuda_fail(cudaErrorMemoryAllocation, "bfs stats buffer");
        rc = bfs_impl(g, root, parent, level, st, as_stream(s));
        if (rc == GB_OK) note_stats_call(st, as_stream(s));
        return rc;
    });
}

gb_status bfs_batch(const gb_graph *g, const int64_t *roots, int k, int32_t *parents,
                    int32_t *levels, gb_stream s)
{
    return guarded([&]() -> gb_status {
        gb_status rc = check_graph(g);
        if (rc != GB_OK) return rc;
        if (!roots || !parents || !levels || k < 1 || k > 64) {
            set_error("bfs_batch: need roots/outputs != NULL and 1 <= k <= 64");
            return GB_ERR_INVALID;
        }
        for (int i = 0; i < k; ++i)
            if (roots[i] < 0 || roots[i] >= g->n) {
                set_error("bfs_batch: a root is outside [0, n)");
                return GB_ERR_RANGE;
            }
        BfsDevStats *st = stats_buffer();
        if (!st) return cuda_fail(cudaErrorMemoryAllocation, "bfs stats buffer");
        rc = msbfs_impl(g, roots, k, parents, levels, st, as_stream(s));
        if (rc == GB_OK) note_stats_call(st, as_stream(s));
        return rc;
    });
}

gb_status bfs_multi_graph(const gb_graph *const *gs, int ng, const int64_t *roots, int r,
                          int32_t *const *parents, int32_t *const *levels, gb_stream s)
{
    return guarded([&]() -> gb_status {
        if (!gs || !roots || !parents || !levels || ng < 1 || ng > 64 || r < 1 || r > 8) {
            set_error("bfs_multi_graph: need arrays != NULL, 1 <= ng <= 64, 1 <= r <= 8");
            return GB_ERR_INVALID;
        }
        for (int i = 0; i < ng; ++i) {
            gb_status rc = check_graph(gs[i]);
            if (rc != GB_OK) return rc;
            if (!parents[i] || !levels[i]) {
                set_error("bfs_multi_graph: NULL output pointer");
                return GB_ERR_INVALID;
            }
            for (int j = 0; j < r; ++j)
                if (roots[(size_t)i * r + j] < 0 || roots[(size_t)i * r + j] >= gs[i]->n) {
                    set_error("bfs_multi_graph: a root is outside [0, n_i)");
                    return GB_ERR_RANGE;
                }
        }
        BfsDevStats *st = stats_buffer();
        if (!st) return cuda_fail(cudaErrorMemoryAllocation, "bfs stats buffer");
        gb_status rc = multigraph_impl(gs, ng, roots, r, parents, levels, st, as_stream(s));
        if (rc == GB_OK) note_stats_call(st, as_stream(s));
        return rc;
    });
}

gb_status bfs_validate(const gb_graph *g, int64_t root, const int32_t *parent,
                       const int32_t *level, const int64_t *edges, int64_t m,
                       gb_validation *out, gb_stream s)
{
    return guarded([&]() -> gb_status {
        if (!g || !parent || !level || !out || m < 0 || (m > 0 && !edges)) {
            set_error("bfs_validate: need g, parent, level, out != NULL, m >= 0, edges != NULL if m > 0");
            return GB_ERR_INVALID;
        }
        return validate_impl(g, root, parent, level, m > 0 ? edges : nullptr, m, out, as_stream(s));
    });
}

gb_status bfs_last_stats(gb_bfs_stats *out)
{
    return guarded([&]() -> gb_status {
        if (!out) {
            set_error("bfs_last_stats: NULL");
            return GB_ERR_INVALID;
        }
        if (!t_stats.valid || !t_stats.dev) {
            set_error("bfs_last_stats: no BFS call on this thread yet");
            return GB_ERR_INVALID;
        }
        BfsDevStats h;
        GB_CUDA(cudaStreamSynchronize(t_stats.stream));
        GB_CUDA(cudaMemcpy(&h, t_stats.dev, sizeof(h), cudaMemcpyDeviceToHost));
        out->nlevels = (int64_t)h.nlevels;
        out->edges_examined = (int64_t)h.edges_examined;
        out->vertices_touched = (int64_t)h.vertices_touched;
        out->reached = (int64_t)h.reached;
        out->td_levels = (int64_t)h.td_levels;
        out->bu_levels = (int64_t)h.bu_levels;
        for (int i = 0; i < GB_STAT_LEVELS; ++i) {
            const bool in = i < kStatLevels && (uint64_t)i < h.nlevels;
            out->level_ns[i] = in ? (int64_t)h.level_ns[i] : 0;
            out->level_frontier[i] = in ? (int64_t)h.level_frontier[i] : 0;
            out->level_dir[i] = in ? h.level_dir[i] : 0;
        }
        return GB_OK;
    });
}

}  // extern "C"
