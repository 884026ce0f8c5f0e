// Serving loop: resident graphs, BFS queries admitted as they arrive and run
// concurrently on the device (continuous batching).
//
// Graphs of 2^14 vertices or more are served by single-source searches: up
// to kPlainSlots queries per graph run at once, each a direction-optimising
// BFS launch on its own stream with an equal share of the SMs, so that the
// searches of all graphs overlap; a query takes the next free slot once its
// output buffers fit in the memory budget.  Measured at 5000 Poisson arrivals
// per second over graphs of SCALE 14-24, this beats both a FIFO of whole-GPU
// searches and multi-source batching: a multi-source level with up to 64 open
// bits scans nearly every edge (its rows rarely complete early), while one
// direction-optimising search touches a small fraction of them.
//
// Smaller graphs keep one multi-source search state (msbfs.cu) whose 64 bits
// are query slots.  A worker thread runs such a graph one BFS level per launch
// on the graph's own stream.  At every level boundary it retires the queries
// whose bit stopped advancing (their BFS is complete), and admits waiting
// queries into free bits as long as their output buffers (8 bytes per vertex)
// fit in the memory budget.  A query admitted at level l starts from its root
// in the frontier of level l; its levels are numbered from there, so its
// result equals a standalone BFS from that root (bits never interact).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gb300bfs.h"
#include "internal.h"

namespace {

double now_s()
{
    using clk = std::chrono::steady_clock;
    return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

enum QState { Q_QUEUED = 0, Q_RUNNING = 1, Q_DONE = 2, Q_RELEASED = 3, Q_CANCELLED = 4 };

constexpr int64_t kPlainMinN = int64_t(1) << 14;  // graphs served one query per launch
constexpr int kPlainSlots = 2;                    // concurrent searches per such graph
constexpr int kMaxPlainSlots = 8;

struct PlainSlot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    gb::BfsDevStats *stats = nullptr;  // device; the kernel's counters land here
    unsigned char *ws = nullptr;       // the slot's own search workspace
    int64_t q = -1;                    // query in flight, -1 if free
};

// Output buffers (parent, level) of one graph, allocated once and reused:
// the serving loop never goes through the stream-ordered allocator.
struct OutBuf {
    int32_t *par = nullptr;
    int32_t *lev = nullptr;
};

struct Query {
    int graph = 0;
    int64_t root = 0;
    double t_arrive = 0;
    double t_done = 0;
    int state = Q_QUEUED;
    bool cancel = false;  // cancelled while running: released as soon as it finishes
    int slot = -1;
    int32_t *par = nullptr;
    int32_t *lev = nullptr;
};

struct GraphRun {
    const gb_graph *g = nullptr;
    gb::MsServe *ms = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    gb::MsCtl *host_ctl = nullptr;  // pinned
    int level = 0;
    unsigned long long active = 0;
    int64_t slot_q[64];
    bool in_flight = false;
    std::deque<int64_t> pending;
    gb::MsSlots slots;
    bool plain = false;  // one query per launch (large graph)
    // counters printed by server_destroy with the verbose option
    int64_t n_launch = 0, n_admit = 0;
    double t_launch = 0, busy_s = 0;
    int plain_blocks = 0;
    PlainSlot ps[kMaxPlainSlots];
    int nplain = 0;  // slots in use
    std::vector<OutBuf> free_out;  // reusable buffers
    std::vector<OutBuf> all_out;   // every buffer ever made (freed at destroy)
};

namespace {
// A free output buffer pair, making one if none is free (synchronous
// cudaMalloc, only while the server grows to its working set).
bool take_out(GraphRun &G, OutBuf &b)
{
    if (!G.free_out.empty()) {
        b = G.free_out.back();
        G.free_out.pop_back();
        return true;
    }
    OutBuf nb;
    if (gb::dmalloc(&nb.par, (size_t)G.g->n * 4) != cudaSuccess) return false;
    if (gb::dmalloc(&nb.lev, (size_t)G.g->n * 4) != cudaSuccess) {
        gb::dfree(nb.par);
        return false;
    }
    G.all_out.push_back(nb);
    b = nb;
    return true;
}
}  // namespace

}  // namespace

struct gb_server {
    int device = 0;
    size_t budget = 0;
    size_t used = 0;        // device bytes counted against the budget: fixed + admitted outputs
    size_t fixed = 0;       // the server's own state (search workspaces, multi-source states)
    gb_server_options opt;
    std::vector<GraphRun> gr;
    std::deque<Query> q;
    std::mutex mu;
    std::condition_variable cv;    // worker wake-up (new work)
    std::condition_variable done;  // a query finished
    std::vector<int64_t> finished;  // tickets finished since the trace runner last looked
    bool tracing = false;           // a trace runner consumes `finished`
    std::thread worker;
    std::atomic<bool> stop{false};
    gb_status fault = GB_OK;
    std::string fault_msg;

    void run();
    bool step_graph(GraphRun &G);
    bool step_plain(GraphRun &G);
    void finish(GraphRun &G, int64_t t, double when);
};

namespace {

size_t out_bytes(const gb_graph *g) { return (size_t)g->n * 8; }

}  // namespace

// A query's search ended (call with mu held): done, or, if it was cancelled
// while running, released at once.
void gb_server::finish(GraphRun &G, int64_t t, double when)
{
    Query &x = q[(size_t)t];
    x.t_done = when;
    x.slot = -1;
    if (x.cancel) {
        G.free_out.push_back(OutBuf{x.par, x.lev});
        x.par = x.lev = nullptr;
        x.state = Q_CANCELLED;
        used -= out_bytes(G.g);
        cv.notify_one();
    } else {
        x.state = Q_DONE;
        if (tracing) finished.push_back(t);
    }
}

// One pass over a large graph: finish completed searches, start new ones in
// free slots while their outputs fit the budget.
bool gb_server::step_plain(GraphRun &G)
{
    bool busy = false;
    for (int i = 0; i < G.nplain; ++i) {
        PlainSlot &P = G.ps[i];
        if (P.q >= 0) {
            const cudaError_t e = cudaEventQuery(P.ev);
            if (e == cudaErrorNotReady) {
                busy = true;
                continue;
            }
            std::lock_guard<std::mutex> lk(mu);
            if (e != cudaSuccess) {
                fault = GB_ERR_CUDA;
                fault_msg = std::string("server search: ") + cudaGetErrorString(e);
                done.notify_all();
                return false;
            }
            finish(G, P.q, now_s());
            P.q = -1;
            done.notify_all();
        }
        // The query's root and buffers are copied out under the lock: other
        // threads append to `q` meanwhile, and no element of it is read
        // without the lock.
        int64_t t = -1, root = 0;
        int32_t *par = nullptr, *lev = nullptr;
        {
            std::lock_guard<std::mutex> lk(mu);
            const size_t need = out_bytes(G.g);
            if (G.pending.empty() || used + need > budget) continue;
            t = G.pending.front();
            Query &x = q[(size_t)t];
            OutBuf ob;
            if (!take_out(G, ob)) continue;  // no device memory now: retry later
            x.par = ob.par;
            x.lev = ob.lev;
            G.pending.pop_front();
            used += need;
            x.state = Q_RUNNING;
            root = x.root;
            par = x.par;
            lev = x.lev;
        }
        ++G.n_launch;
        ++G.n_admit;
        gb_status rc = gb::bfs_impl(G.g, root, par, lev, P.stats, P.stream, G.plain_blocks, P.ws);
        if (rc == GB_OK && cudaEventRecord(P.ev, P.stream) != cudaSuccess) rc = GB_ERR_CUDA;
        if (rc != GB_OK) {
            std::lock_guard<std::mutex> lk(mu);
            fault = rc;
            fault_msg = gb::last_error();
            done.notify_all();
            return false;
        }
        P.q = t;
        busy = true;
    }
    return busy;
}

// One pass over a graph: collect a finished level, retire, admit, launch the
// next level.  Returns true if the graph has work in flight.
bool gb_server::step_graph(GraphRun &G)
{
    if (G.plain) return step_plain(G);
    if (G.in_flight) {
        const cudaError_t e = cudaEventQuery(G.ev);
        if (e == cudaErrorNotReady) return true;
        G.in_flight = false;
        if (e != cudaSuccess) {
            std::lock_guard<std::mutex> lk(mu);
            fault = GB_ERR_CUDA;
            fault_msg = std::string("server level: ") + cudaGetErrorString(e);
            done.notify_all();
            return false;
        }
        const unsigned long long adv = G.host_ctl->anynew;
        const double t = now_s();
        G.busy_s += t - G.t_launch;
        std::lock_guard<std::mutex> lk(mu);
        for (int b = 0; b < 64; ++b) {
            const unsigned long long bit = 1ull << b;
            if ((G.active & bit) && !(adv & bit)) {  // nothing new: this BFS is complete
                finish(G, G.slot_q[b], t);
                G.active &= ~bit;
                G.slot_q[b] = -1;
            }
        }
        ++G.level;
        done.notify_all();
    }
    // admissions at this level boundary
    int nadm = 0;
    int bits[64];
    int64_t roots[64];
    {
        std::lock_guard<std::mutex> lk(mu);
        const size_t need = out_bytes(G.g);
        while (!G.pending.empty() && G.active != ~0ull && used + need <= budget) {
            const int64_t t = G.pending.front();
            Query &x = q[(size_t)t];
            int b = 0;
            while ((G.active >> b) & 1ull) ++b;
            OutBuf ob;
            if (!take_out(G, ob)) break;  // no device memory now: retry at the next boundary
            x.par = ob.par;
            x.lev = ob.lev;
            G.pending.pop_front();
            used += need;
            cudaMemsetAsync(x.par, 0xff, (size_t)G.g->n * 4, G.stream);  // -1 everywhere
            cudaMemsetAsync(x.lev, 0xff, (size_t)G.g->n * 4, G.stream);
            x.state = Q_RUNNING;
            x.slot = b;
            G.active |= 1ull << b;
            G.slot_q[b] = t;
            G.slots.par[b] = x.par;
            G.slots.lev[b] = x.lev;
            G.slots.start[b] = G.level;
            bits[nadm] = b;
            roots[nadm] = x.root;
            ++nadm;
        }
    }
    gb_status rc = GB_OK;
    if (nadm) rc = gb::ms_serve_admit(G.ms, G.level, nadm, bits, roots, &G.slots, G.stream);
    G.n_admit += nadm;
    if (rc == GB_OK && G.active) {
        G.t_launch = now_s();
        ++G.n_launch;
        rc = gb::ms_serve_step(G.ms, G.level, G.active, G.host_ctl, G.stream);
        if (rc == GB_OK && cudaEventRecord(G.ev, G.stream) != cudaSuccess) rc = GB_ERR_CUDA;
        if (rc == GB_OK) G.in_flight = true;
    }
    if (rc != GB_OK) {
        std::lock_guard<std::mutex> lk(mu);
        fault = rc;
        fault_msg = gb::last_error();
        done.notify_all();
        return false;
    }
    return G.in_flight;
}

void gb_server::run()
{
    cudaSetDevice(device);
    int64_t iters = 0;
    const double t_start = now_s();
    while (!stop.load()) {
        ++iters;
        bool busy = false;
        for (auto &G : gr) busy |= step_graph(G);
        {
            std::unique_lock<std::mutex> lk(mu);
            if (fault != GB_OK) break;
            bool waiting = false;
            for (auto &G : gr) waiting |= !G.pending.empty();
            if (!busy && !waiting) cv.wait_for(lk, std::chrono::microseconds(200));
        }
        if (busy) std::this_thread::yield();
    }
    if (opt.verbose) {
        std::fprintf(stderr, "[server] worker iterations %lld over %.3f s\n", (long long)iters,
                     now_s() - t_start);
        for (size_t i = 0; i < gr.size(); ++i)
            std::fprintf(stderr, "[server] graph %zu n=%lld %s launches %lld admits %lld busy %.3f s\n",
                         i, (long long)gr[i].g->n, gr[i].plain ? "single" : "batched",
                         (long long)gr[i].n_launch, (long long)gr[i].n_admit, gr[i].busy_s);
    }
}

extern "C" {

gb_status server_default_options(gb_server_options *out)
{
    if (!out) {
        gb::set_error("server_default_options: NULL");
        return GB_ERR_INVALID;
    }
    out->single_source_min_vertices = kPlainMinN;
    out->slots_per_graph = kPlainSlots;
    out->full_grid = 0;
    out->verbose = 0;
    return GB_OK;
}

gb_status server_create(const gb_graph *const *gs, int ng, size_t mem_budget, gb_server **out)
{
    gb_server_options o;
    server_default_options(&o);
    return server_create_with_options(gs, ng, mem_budget, &o, out);
}

gb_status server_create_with_options(const gb_graph *const *gs, int ng, size_t mem_budget,
                                     const gb_server_options *opt, gb_server **out)
{
    if (!out || !gs || ng < 1 || !opt) {
        gb::set_error("server_create: need graphs, options and out");
        return GB_ERR_INVALID;
    }
    if (opt->slots_per_graph < 1 || opt->slots_per_graph > kMaxPlainSlots ||
        opt->single_source_min_vertices < 0) {
        gb::set_error("server_create: slots_per_graph must be 1..8 and single_source_min_vertices >= 0");
        return GB_ERR_INVALID;
    }
    *out = nullptr;
    gb::Context *ctx = gb::context();
    if (!ctx) return GB_ERR_CUDA;
    gb_server *srv = new gb_server();
    srv->device = ctx->device;
    srv->budget = mem_budget;
    srv->opt = *opt;
    srv->gr.resize(ng);
    const int64_t plain_min = opt->single_source_min_vertices;
    const int nplain = opt->slots_per_graph;
    const bool full_grid = opt->full_grid != 0;
    int64_t ntot = 0;  // vertices of the graphs batched as bits (the small ones)
    for (int i = 0; i < ng; ++i) ntot += (gs[i] && gs[i]->n < plain_min) ? gs[i]->n : 0;
    gb_status rc = GB_OK;
    for (int i = 0; i < ng && rc == GB_OK; ++i) {
        GraphRun &G = srv->gr[i];
        if (!gs[i] || !gs[i]->off) {
            gb::set_error("server_create: NULL graph");
            rc = GB_ERR_INVALID;
            break;
        }
        G.g = gs[i];
        for (int b = 0; b < 64; ++b) {
            G.slot_q[b] = -1;
            G.slots.par[b] = nullptr;
            G.slots.lev[b] = nullptr;
            G.slots.start[b] = 0;
        }
        if (G.g->n >= plain_min) {
            G.plain = true;
            G.nplain = nplain;
            G.plain_blocks = full_grid ? ctx->bfs_blocks2 : std::max(8, ctx->bfs_blocks2 / nplain);
            for (int k = 0; k < nplain && rc == GB_OK; ++k) {
                PlainSlot &P = G.ps[k];
                cudaError_t e = cudaSuccess;
                if ((e = cudaStreamCreateWithFlags(&P.stream, cudaStreamNonBlocking)) != cudaSuccess ||
                    (e = cudaEventCreateWithFlags(&P.ev, cudaEventDisableTiming)) != cudaSuccess ||
                    (e = gb::dmalloc(&P.stats, sizeof(gb::BfsDevStats))) != cudaSuccess ||
                    (e = gb::dmalloc(&P.ws, gb::bfs_workspace_bytes(G.g))) != cudaSuccess) {
                    rc = gb::cuda_fail(e, "server_create: slot stream, event or workspace");
                }
                srv->fixed += sizeof(gb::BfsDevStats) + gb::bfs_workspace_bytes(G.g);
            }
            continue;
        }
        // every batched graph gets a share of the GPU proportional to its
        // size among the batched graphs, so that their levels run side by side
        const int blocks = full_grid ? ctx->ms_blocks
                                     : (int)std::max<int64_t>(
                                           8, (int64_t)ctx->ms_blocks * G.g->n / std::max<int64_t>(ntot, 1));
        if (cudaStreamCreateWithFlags(&G.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&G.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost((void **)&G.host_ctl, sizeof(gb::MsCtl)) != cudaSuccess) {
            gb::set_error("server_create: stream/event/pinned buffer");
            rc = GB_ERR_CUDA;
            break;
        }
        rc = gb::ms_serve_create(G.g, blocks, &G.ms, G.stream);
        if (rc == GB_OK) srv->fixed += gb::ms_serve_bytes(G.ms);
    }
    if (rc == GB_OK && srv->fixed > mem_budget) {
        gb::set_error("server_create: the memory budget (" + std::to_string(mem_budget) +
                      " bytes) does not hold the server's own search state (" +
                      std::to_string(srv->fixed) + " bytes)");
        rc = GB_ERR_NOMEM;
    }
    srv->used = srv->fixed;
    if (rc != GB_OK) {
        for (auto &G : srv->gr) {
            for (auto &P : G.ps) {
                if (P.ws) gb::dfree(P.ws);
                if (P.stats) gb::dfree(P.stats);
                if (P.ev) cudaEventDestroy(P.ev);
                if (P.stream) cudaStreamDestroy(P.stream);
            }
            if (G.ms) gb::ms_serve_destroy(G.ms);
            if (G.ev) cudaEventDestroy(G.ev);
            if (G.stream) cudaStreamDestroy(G.stream);
            if (G.host_ctl) cudaFreeHost(G.host_ctl);
        }
        delete srv;
        return rc;
    }
    srv->worker = std::thread([srv]() { srv->run(); });
    *out = srv;
    return GB_OK;
}

gb_status server_submit(gb_server *srv, int graph_id, int64_t root, int64_t *ticket)
{
    if (!srv || !ticket) {
        gb::set_error("server_submit: NULL");
        return GB_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->fault != GB_OK) {
        gb::set_error(srv->fault_msg);
        return srv->fault;
    }
    if (graph_id < 0 || graph_id >= (int)srv->gr.size() || root < 0 ||
        root >= srv->gr[graph_id].g->n) {
        gb::set_error("server_submit: graph or root out of range");
        return GB_ERR_RANGE;
    }
    Query x;
    x.graph = graph_id;
    x.root = root;
    x.t_arrive = now_s();
    srv->q.push_back(x);
    *ticket = (int64_t)srv->q.size() - 1;
    srv->gr[graph_id].pending.push_back(*ticket);
    srv->cv.notify_one();
    return GB_OK;
}

gb_status server_poll(gb_server *srv, int64_t ticket, const int32_t **parent,
                      const int32_t **level)
{
    if (!srv) return GB_ERR_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->fault != GB_OK) {
        gb::set_error(srv->fault_msg);
        return srv->fault;
    }
    if (ticket < 0 || ticket >= (int64_t)srv->q.size()) {
        gb::set_error("server_poll: unknown ticket");
        return GB_ERR_INVALID;
    }
    const Query &x = srv->q[(size_t)ticket];
    if (x.state == Q_RELEASED || x.state == Q_CANCELLED || x.cancel) {
        gb::set_error(x.state == Q_RELEASED ? "server_poll: ticket already released"
                                            : "server_poll: query cancelled");
        return GB_ERR_INVALID;
    }
    if (x.state != Q_DONE) return GB_ERR_BUSY;
    if (parent) *parent = x.par;
    if (level) *level = x.lev;
    return GB_OK;
}

gb_status server_release(gb_server *srv, int64_t ticket)
{
    if (!srv) return GB_ERR_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (ticket < 0 || ticket >= (int64_t)srv->q.size()) {
        gb::set_error("server_release: unknown ticket");
        return GB_ERR_INVALID;
    }
    Query &x = srv->q[(size_t)ticket];
    if (x.state != Q_DONE) {
        gb::set_error("server_release: query not finished");
        return GB_ERR_BUSY;
    }
    GraphRun &G = srv->gr[x.graph];
    G.free_out.push_back(OutBuf{x.par, x.lev});
    x.par = x.lev = nullptr;
    x.state = Q_RELEASED;
    srv->used -= out_bytes(G.g);
    srv->cv.notify_one();
    return GB_OK;
}

gb_status server_cancel(gb_server *srv, int64_t ticket)
{
    if (!srv) return GB_ERR_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (ticket < 0 || ticket >= (int64_t)srv->q.size()) {
        gb::set_error("server_cancel: unknown ticket");
        return GB_ERR_INVALID;
    }
    Query &x = srv->q[(size_t)ticket];
    GraphRun &G = srv->gr[x.graph];
    switch (x.state) {
    case Q_QUEUED: {
        auto it = std::find(G.pending.begin(), G.pending.end(), ticket);
        if (it != G.pending.end()) G.pending.erase(it);
        x.state = Q_CANCELLED;
        return GB_OK;
    }
    case Q_RUNNING:
        if (x.cancel) break;
        x.cancel = true;  // its search runs out; finish() releases it
        return GB_OK;
    case Q_DONE:
        G.free_out.push_back(OutBuf{x.par, x.lev});
        x.par = x.lev = nullptr;
        x.state = Q_CANCELLED;
        srv->used -= out_bytes(G.g);
        srv->cv.notify_one();
        return GB_OK;
    default:
        break;
    }
    gb::set_error("server_cancel: query already released or cancelled");
    return GB_ERR_INVALID;
}

gb_status server_stats(gb_server *srv, gb_server_stats *out)
{
    if (!srv || !out) {
        gb::set_error("server_stats: NULL");
        return GB_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = gb_server_stats{};
    out->budget_bytes = (int64_t)srv->budget;
    out->fixed_bytes = (int64_t)srv->fixed;
    out->used_bytes = (int64_t)srv->used;
    for (const Query &x : srv->q) {
        if (x.state == Q_QUEUED) ++out->queued;
        else if (x.state == Q_RUNNING) ++out->running;
        else if (x.state == Q_DONE) ++out->done;
        else if (x.state == Q_RELEASED) ++out->released;
        else if (x.state == Q_CANCELLED) ++out->cancelled;
    }
    return GB_OK;
}

gb_status server_run_trace(gb_server *srv, int64_t nq, const double *t_arrival_s,
                           const int32_t *graph_id, const int64_t *root, int keep_results,
                           double *latency_ms)
{
    if (!srv || nq < 0 || (nq > 0 && (!t_arrival_s || !graph_id || !root || !latency_ms))) {
        gb::set_error("server_run_trace: bad arguments");
        return GB_ERR_INVALID;
    }
    std::vector<int64_t> tickets((size_t)nq, -1);
    std::unordered_map<int64_t, int64_t> index;  // ticket -> position in the trace
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->finished.clear();
        srv->tracing = true;
    }
    struct TraceEnd {
        gb_server *s;
        ~TraceEnd()
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->tracing = false;
            s->finished.clear();
        }
    } trace_end{srv};
    const double t0 = now_s();
    int64_t next = 0, nfin = 0;
    std::unique_lock<std::mutex> lk(srv->mu);
    while (nfin < nq) {
        if (srv->fault != GB_OK) {
            gb::set_error(srv->fault_msg);
            return srv->fault;
        }
        // submit every query that has arrived, stamped with its arrival time
        const double t = now_s();
        bool submitted = false;
        while (next < nq && t0 + t_arrival_s[next] <= t) {
            const int gid = graph_id[next];
            if (gid < 0 || gid >= (int)srv->gr.size() || root[next] < 0 ||
                root[next] >= srv->gr[gid].g->n) {
                gb::set_error("server_run_trace: graph or root out of range");
                return GB_ERR_RANGE;
            }
            Query x;
            x.graph = gid;
            x.root = root[next];
            x.t_arrive = t0 + t_arrival_s[next];
            srv->q.push_back(x);
            tickets[(size_t)next] = (int64_t)srv->q.size() - 1;
            index[tickets[(size_t)next]] = next;
            srv->gr[gid].pending.push_back(tickets[(size_t)next]);
            ++next;
            submitted = true;
        }
        if (submitted) srv->cv.notify_one();
        // record and release the finished ones, so their memory admits new queries
        std::vector<int64_t> got;
        got.swap(srv->finished);
        for (const int64_t tk : got) {
            const auto it = index.find(tk);
            if (it == index.end()) continue;  // a query submitted outside this trace
            const int64_t i = it->second;
            Query &x = srv->q[(size_t)tk];
            ++nfin;
            latency_ms[i] = (x.t_done - x.t_arrive) * 1e3;
            if (!keep_results) {
                GraphRun &G = srv->gr[x.graph];
                G.free_out.push_back(OutBuf{x.par, x.lev});
                x.par = x.lev = nullptr;
                x.state = Q_RELEASED;
                srv->used -= out_bytes(G.g);
            }
        }
        if (!got.empty()) srv->cv.notify_one();
        if (nfin >= nq) break;
        // sleep until the next arrival or a completion, whichever comes first
        double wait = 1e-3;
        if (next < nq) wait = std::min(wait, std::max(0.0, t0 + t_arrival_s[next] - now_s()));
        if (wait > 20e-6) srv->done.wait_for(lk, std::chrono::duration<double>(wait));
        else {
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        }
    }
    return GB_OK;
}

gb_status server_destroy(gb_server *srv)
{
    if (!srv) return GB_OK;
    srv->stop.store(true);
    srv->cv.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    cudaSetDevice(srv->device);
    for (auto &G : srv->gr) {
        if (G.stream) cudaStreamSynchronize(G.stream);
        for (auto &P : G.ps)
            if (P.stream) cudaStreamSynchronize(P.stream);
    }
    for (auto &G : srv->gr) {
        for (auto &b : G.all_out) {
            gb::dfree(b.par);
            gb::dfree(b.lev);
        }
        for (auto &P : G.ps) {
            if (P.ws) gb::dfree(P.ws);
            if (P.stats) gb::dfree(P.stats);
            if (P.ev) cudaEventDestroy(P.ev);
            if (P.stream) cudaStreamDestroy(P.stream);
        }
        if (G.ms) gb::ms_serve_destroy(G.ms);
        if (G.ev) cudaEventDestroy(G.ev);
        if (G.stream) cudaStreamDestroy(G.stream);
        if (G.host_ctl) cudaFreeHost(G.host_ctl);
    }
    delete srv;
    return GB_OK;
}

}  // extern "C"
