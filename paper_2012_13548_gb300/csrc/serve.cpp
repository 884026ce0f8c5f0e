// Serving loop: resident graphs, BFS queries admitted as they arrive
// (continuous batching at level granularity).
//
// Every resident graph keeps one multi-source search state (msbfs.cu) whose
// 64 bits are query slots.  A worker thread runs each graph one BFS level per
// launch on the graph's own stream.  At every level boundary it retires the
// queries whose bit stopped advancing (their BFS is complete), and admits
// waiting queries into free bits as long as their output buffers (8 bytes per
// vertex) fit in the memory budget.  A query admitted at level l starts from
// its root in the frontier of level l; its levels are numbered from there, so
// its result equals a standalone BFS from that root (bits never interact).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "gb300bfs.h"
#include "internal.h"

namespace {

double now_s()
{
    using clk = std::chrono::steady_clock;
    return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

enum QState { Q_QUEUED = 0, Q_RUNNING = 1, Q_DONE = 2, Q_RELEASED = 3 };

struct Query {
    int graph = 0;
    int64_t root = 0;
    double t_arrive = 0;
    double t_done = 0;
    int state = Q_QUEUED;
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
};

}  // namespace

struct gb_server {
    int device = 0;
    size_t budget = 0;
    size_t used = 0;
    std::vector<GraphRun> gr;
    std::deque<Query> q;
    std::mutex mu;
    std::condition_variable cv;    // worker wake-up (new work)
    std::condition_variable done;  // a query finished
    std::thread worker;
    std::atomic<bool> stop{false};
    gb_status fault = GB_OK;
    std::string fault_msg;

    void run();
    bool step_graph(GraphRun &G);
};

namespace {

size_t out_bytes(const gb_graph *g) { return (size_t)g->n * 8; }

}  // namespace

// One pass over a graph: collect a finished level, retire, admit, launch the
// next level.  Returns true if the graph has work in flight.
bool gb_server::step_graph(GraphRun &G)
{
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
        std::lock_guard<std::mutex> lk(mu);
        for (int b = 0; b < 64; ++b) {
            const unsigned long long bit = 1ull << b;
            if ((G.active & bit) && !(adv & bit)) {  // nothing new: this BFS is complete
                Query &x = q[(size_t)G.slot_q[b]];
                x.state = Q_DONE;
                x.t_done = t;
                x.slot = -1;
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
            if (cudaMallocAsync((void **)&x.par, (size_t)G.g->n * 4, G.stream) != cudaSuccess ||
                cudaMallocAsync((void **)&x.lev, (size_t)G.g->n * 4, G.stream) != cudaSuccess) {
                if (x.par) cudaFreeAsync(x.par, G.stream);
                x.par = nullptr;
                x.lev = nullptr;
                break;  // no device memory now: retry at the next boundary
            }
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
    if (rc == GB_OK && G.active) {
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
    while (!stop.load()) {
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
}

extern "C" {

gb_status server_create(const gb_graph *const *gs, int ng, size_t mem_budget, gb_server **out)
{
    if (!out || !gs || ng < 1) {
        gb::set_error("server_create: need graphs and out");
        return GB_ERR_INVALID;
    }
    *out = nullptr;
    gb::Context *ctx = gb::context();
    if (!ctx) return GB_ERR_CUDA;
    gb_server *srv = new gb_server();
    srv->device = ctx->device;
    srv->budget = mem_budget;
    srv->gr.resize(ng);
    int64_t ntot = 0;
    for (int i = 0; i < ng; ++i) ntot += gs[i] ? gs[i]->n : 0;
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
        // every graph gets a share of the GPU proportional to its size, so
        // that the levels of several graphs run side by side
        const int blocks = (int)std::max<int64_t>(
            8, (int64_t)ctx->ms_blocks * G.g->n / std::max<int64_t>(ntot, 1));
        if (cudaStreamCreateWithFlags(&G.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&G.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost((void **)&G.host_ctl, sizeof(gb::MsCtl)) != cudaSuccess) {
            gb::set_error("server_create: stream/event/pinned buffer");
            rc = GB_ERR_CUDA;
            break;
        }
        rc = gb::ms_serve_create(G.g, blocks, &G.ms, G.stream);
    }
    if (rc != GB_OK) {
        for (auto &G : srv->gr) {
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
    if (x.state == Q_RELEASED) {
        gb::set_error("server_poll: ticket already released");
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
    cudaFreeAsync(x.par, G.stream);
    cudaFreeAsync(x.lev, G.stream);
    x.par = x.lev = nullptr;
    x.state = Q_RELEASED;
    srv->used -= out_bytes(G.g);
    srv->cv.notify_one();
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
    const double t0 = now_s();
    int64_t next = 0;
    while (next < nq) {
        const double due = t0 + t_arrival_s[next];
        double t = now_s();
        if (t < due) {
            if (due - t > 200e-6)
                std::this_thread::sleep_for(std::chrono::duration<double>(due - t - 100e-6));
            continue;
        }
        // submit every query that has arrived, stamped with its arrival time
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->fault != GB_OK) {
            gb::set_error(srv->fault_msg);
            return srv->fault;
        }
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
            srv->gr[gid].pending.push_back(tickets[(size_t)next]);
            ++next;
        }
        srv->cv.notify_one();
    }
    // wait for all of them, releasing results as they finish
    int64_t finished = 0;
    std::vector<char> seen((size_t)nq, 0);
    std::unique_lock<std::mutex> lk(srv->mu);
    while (finished < nq) {
        if (srv->fault != GB_OK) {
            gb::set_error(srv->fault_msg);
            return srv->fault;
        }
        for (int64_t i = 0; i < nq; ++i) {
            if (seen[(size_t)i]) continue;
            Query &x = srv->q[(size_t)tickets[(size_t)i]];
            if (x.state != Q_DONE) continue;
            seen[(size_t)i] = 1;
            ++finished;
            latency_ms[i] = (x.t_done - x.t_arrive) * 1e3;
            if (!keep_results) {
                GraphRun &G = srv->gr[x.graph];
                cudaFreeAsync(x.par, G.stream);
                cudaFreeAsync(x.lev, G.stream);
                x.par = x.lev = nullptr;
                x.state = Q_RELEASED;
                srv->used -= out_bytes(G.g);
                srv->cv.notify_one();
            }
        }
        if (finished < nq) srv->done.wait_for(lk, std::chrono::milliseconds(1));
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
    for (auto &x : srv->q) {
        cudaStream_t st = srv->gr[x.graph].stream;
        if (x.par) cudaFreeAsync(x.par, st);
        if (x.lev) cudaFreeAsync(x.lev, st);
    }
    for (auto &G : srv->gr) {
        if (G.stream) cudaStreamSynchronize(G.stream);
    }
    for (auto &G : srv->gr) {
        if (G.ms) gb::ms_serve_destroy(G.ms);
        if (G.ev) cudaEventDestroy(G.ev);
        if (G.stream) cudaStreamDestroy(G.stream);
        if (G.host_ctl) cudaFreeHost(G.host_ctl);
    }
    delete srv;
    return GB_OK;
}

}  // extern "C"
