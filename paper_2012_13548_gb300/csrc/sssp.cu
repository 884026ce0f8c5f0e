// Kernel 3 (Sec. 2.4): single-source shortest paths on the weighted graph.
//
// The paper states Dijkstra's algorithm (Algorithm "Sequential SSSP": take the
// closest vertex left, relax its edges) and names delta-stepping as the
// parallel route (Sec. 4.1).  This is delta-stepping in its near/far form, run
// by one persistent cooperative kernel:
//
//   * distances are 64-bit integers in units of 2^-24 (every weight is a
//     multiple of 2^-24 in (0, 1]), so a relaxation is an exact integer add
//     and an atomic minimum, and the distances are those of the rounding-free
//     Dijkstra;
//   * the current bucket holds the distances below the threshold T.  The
//     near queue lists the vertices to expand; an expansion that lowers a
//     neighbour below T queues it for the next round (once per round, by a
//     stamp), one that lowers it to T or more lists it as far (once per
//     bucket);
//   * when a round leaves the near queue empty, every distance below T is
//     final.  The least far distance d at or above T picks the next bucket,
//     T = (d / delta + 1) * delta (empty buckets are skipped), and the far
//     list is split: entries below T (settled meanwhile) are dropped, entries
//     inside the new bucket form the near queue, the rest the next far list;
//   * light and heavy edges (Meyer and Sanders' split, taken per vertex): the
//     search reads a second copy of every row sorted by weight.  Expanding u
//     relaxes only the prefix of its row with w < T - dist(u), the edges that
//     can still land in the current bucket; u is listed once per bucket, and
//     when the bucket is settled the rest of each listed row (the heavy
//     edges, which can only produce distances >= T) is relaxed once, with
//     the final dist(u).  A vertex expanded again after its distance dropped
//     re-reads only its light prefix;
//   * rows longer than SP_BIG are cut into SP_CHUNK-edge chunks that all warps
//     share (a chunk tests each edge against the split itself); shorter rows
//     find their split by bisection and are expanded 32 per warp as one
//     stream of edges;
//   * a relaxation that lowers dist(v) also writes u as v's parent (a plain
//     store: racing winners may leave a parent that is no longer tight);
//   * after the last bucket the kernel writes the distances as doubles and the
//     tree: by default each recorded parent is checked (one bisection of v's
//     row) and kept if tight, dist(u) + w(u,v) = dist(v); otherwise, and for
//     every vertex in canonical mode, parent(v) is the smallest-id tight
//     neighbour, the first tight entry of v's column-sorted row.
//
// Kernel 1's weights: graph_build_csr_weighted builds the CSR as kernel 1 does
// and then gives each entry the least weight among the tuples joining its pair
// (each tuple finds its two entries by bisection of the sorted rows); the
// weight-sorted rows come from one radix sort of (row << 25 | weight) keys
// carrying the columns (stable, so equal weights keep ascending columns).
#include "common.cuh"
#include "internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace gb {
namespace {

constexpr int SP_THREADS = 512;
constexpr int SP_MINB = 2;
constexpr int64_t SP_BIG = 1024;   // longer rows are expanded in chunks by all warps
constexpr int64_t SP_CHUNK = 256;  // edges per chunk
constexpr unsigned long long SP_INF = ~0ull;
constexpr double kUnit = 5.9604644775390625e-8;  // 2^-24: one weight unit
constexpr int SITE_SP_BAR = 40, SITE_SP_NEAR = 41, SITE_SP_FAR = 42, SITE_SP_BIGQ = 43,
              SITE_SP_ROUNDS = 44, SITE_SP_W = 45, SITE_SP_FIND = 46;

// ---------------------------------------------------------------------------
// Kernel 1's weights
// ---------------------------------------------------------------------------

// Weight w in (0, 1] as units of 2^-24, rounded to the nearest unit and at
// least one; 0 for a weight outside (0, 1] or NaN.
__device__ __forceinline__ uint32_t weight_units(float w)
{
    if (!(w > 0.0f && w <= 1.0f)) return 0u;
    const uint32_t k = __float2uint_rn(w * 16777216.0f);
    return k < 1u ? 1u : k;
}

// Index of column v in the sorted row [lo, hi), or -1.
__device__ __forceinline__ int64_t find_in_row(const int32_t *__restrict__ col, int64_t lo, int64_t hi,
                                               int32_t v)
{
    const int64_t end = hi;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo < end && col[lo] == v ? lo : -1;
}

__global__ void wt_attach_kernel(const int64_t *__restrict__ edges, const float *__restrict__ w,
                                 int64_t m, const int64_t *__restrict__ off,
                                 const int32_t *__restrict__ col, int64_t n,
                                 uint32_t *__restrict__ wgt, DevStatus *st)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int64_t u = edges[e], v = edges[m + e];
        const uint32_t k = weight_units(w[e]);
        if (k == 0u) {
            record_error(st, GB_ERR_RANGE, SITE_SP_W, (long long)e);
            continue;
        }
        if (u < 0 || u >= n || v < 0 || v >= n || u == v) continue;  // range: kernel 1 reported it
        const int64_t j1 = find_in_row(col, off[u], off[u + 1], (int32_t)v);
        const int64_t j2 = find_in_row(col, off[v], off[v + 1], (int32_t)u);
        if (j1 < 0 || j2 < 0) {
            record_error(st, GB_ERR_RANGE, SITE_SP_FIND, (long long)e);
            continue;
        }
        atomicMin(&wgt[j1], k);
        atomicMin(&wgt[j2], k);
    }
}

// Keys (row << 25 | weight) and column values of every entry, one warp per row.
__global__ void wsort_keys_kernel(const int64_t *__restrict__ off, const int32_t *__restrict__ col,
                                  const uint32_t *__restrict__ wgt, int64_t n,
                                  uint64_t *__restrict__ keys, uint32_t *__restrict__ vals)
{
    const unsigned lane = threadIdx.x & 31u;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = gwarp; u < n; u += nwarps) {
        const int64_t s0 = off[u], e0 = off[u + 1];
        for (int64_t j = s0 + lane; j < e0; j += 32) {
            keys[j] = ((uint64_t)u << 25) | (uint64_t)wgt[j];
            vals[j] = (uint32_t)col[j];
        }
    }
}

__global__ void wsort_pack_kernel(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                                  int64_t nnz, uint2 *__restrict__ wadj)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz; j += stride)
        wadj[j] = make_uint2(vals[j], (uint32_t)(keys[j] & 0x1ffffffull));
}

// ---------------------------------------------------------------------------
// The search
// ---------------------------------------------------------------------------

struct SpBig {
    int32_t u;
    uint32_t cbase;  // first chunk of the row in the queue's chunk numbering
};

struct SpQueueCtl {
    unsigned long long cnt;  // vertices in the queue
    unsigned long long big;  // (big rows << 32) | their chunks
};

struct SpHeader {
    GridBarrier bar;
    unsigned long long minfar;     // least far distance >= T (bucket advance)
    unsigned long long farcnt[2];  // far list sizes, by epoch parity
    SpQueueCtl q[4];               // near queue counters, by queue id mod 4
    SpQueueCtl settle;             // vertices expanded in the current bucket
    unsigned long long acc[4];     // processed, scanned, won, reached
};

struct SpArgs {
    const int64_t *off;
    const int32_t *col;
    const uint32_t *wgt;
    const uint2 *wadj;         // rows by ascending weight: (column, weight)
    int64_t n;
    int32_t root;
    unsigned long long *dist;  // [n] units of 2^-24, SP_INF if unreached
    uint32_t *nstamp;          // [n] id of the last near queue v entered
    uint32_t *fstamp;          // [n] epoch of the last far list v entered
    uint32_t *sstamp;          // [n] epoch of the bucket that expanded v
    int32_t *nq;               // 2 near queues of n
    int32_t *fq;               // 2 far lists of n
    int32_t *sq;               // the settle list of n
    SpBig *bq;                 // 2 big-row lists of bigcap, then the settle list's
    int64_t bigcap;
    SpHeader *hdr;
    DevStatus *st;
    SsspDevStats *stats;
    unsigned long long delta;
    double *dist_out;
    int32_t *parent;
    int canonical;  // 1: the smallest-id tight parent of every vertex
    uint64_t timeout_ns;
    uint64_t run_limit_ns;  // the search gives up (GB_ERR_TIMEOUT) after this long
    long long max_rounds;
};

__device__ __forceinline__ SpBig load_spbig(const SpBig *q, int64_t i)
{
    const unsigned long long r = __ldcg(reinterpret_cast<const unsigned long long *>(q) + i);
    SpBig b;
    b.u = (int32_t)(r & 0xffffffffull);
    b.cbase = (uint32_t)(r >> 32);
    return b;
}

// Warp-collective: the lanes with `want` append v to near queue `qid`; a row
// longer than SP_BIG is also listed with its chunks.
__device__ __forceinline__ void push_near(const SpArgs &a, unsigned qid, bool want, int32_t v)
{
    const unsigned m = __ballot_sync(kFull, want);
    if (!m) return;
    const unsigned lane = lane_id();
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if ((int)lane == leader) base = atomicAdd(&a.hdr->q[qid & 3].cnt, (unsigned long long)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (!want) return;
    const int64_t pos = (int64_t)base + __popc(m & lanemask_lt());
    if (pos < a.n) a.nq[(int64_t)(qid & 1) * a.n + pos] = v;
    else record_error(a.st, GB_ERR_RANGE, SITE_SP_NEAR, pos);
    const int64_t d = a.off[v + 1] - a.off[v];
    if (d > SP_BIG) {
        const unsigned nch = (unsigned)((d + SP_CHUNK - 1) / SP_CHUNK);
        const unsigned long long old = atomicAdd(&a.hdr->q[qid & 3].big, (1ull << 32) | nch);
        const int64_t bi = (int64_t)(old >> 32);
        if (bi < a.bigcap) {
            const unsigned long long r = (unsigned long long)(uint32_t)v | ((old & 0xffffffffull) << 32);
            reinterpret_cast<unsigned long long *>(a.bq)[(int64_t)(qid & 1) * a.bigcap + bi] = r;
        } else {
            record_error(a.st, GB_ERR_RANGE, SITE_SP_BIGQ, bi);
        }
    }
}

// Warp-collective: the lanes with `want` append v to the settle list of the
// current bucket (a row longer than SP_BIG also with its chunks).
__device__ __forceinline__ void push_settle(const SpArgs &a, bool want, int32_t v, int64_t d)
{
    const unsigned m = __ballot_sync(kFull, want);
    if (!m) return;
    const unsigned lane = lane_id();
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if ((int)lane == leader) base = atomicAdd(&a.hdr->settle.cnt, (unsigned long long)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (!want) return;
    const int64_t pos = (int64_t)base + __popc(m & lanemask_lt());
    if (pos < a.n) a.sq[pos] = v;
    else record_error(a.st, GB_ERR_RANGE, SITE_SP_NEAR, pos);
    if (d > SP_BIG) {
        const unsigned nch = (unsigned)((d + SP_CHUNK - 1) / SP_CHUNK);
        const unsigned long long old = atomicAdd(&a.hdr->settle.big, (1ull << 32) | nch);
        const int64_t bi = (int64_t)(old >> 32);
        if (bi < a.bigcap) {
            const unsigned long long r = (unsigned long long)(uint32_t)v | ((old & 0xffffffffull) << 32);
            reinterpret_cast<unsigned long long *>(a.bq)[2 * a.bigcap + bi] = r;
        } else {
            record_error(a.st, GB_ERR_RANGE, SITE_SP_BIGQ, bi);
        }
    }
}

// The weight-sorted rows are a stream (each entry read about once by a light
// prefix and once by a settle step): they are loaded with an L2 evict-first
// policy and no L1 allocation, so that they do not push the distance array
// and the stamps, which every relaxation reads at random, out of L2.
__device__ __forceinline__ uint64_t stream_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ uint2 ld_stream(const uint2 *p, uint64_t pol)
{
    uint2 r;
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
                 : "=r"(r.x), "=r"(r.y)
                 : "l"(p), "l"(pol));
    return r;
}

// First index j in [lo, hi) of a weight-sorted row with weight >= lim (hi if none).
__device__ __forceinline__ int64_t weight_split(const uint2 *__restrict__ wadj, int64_t lo, int64_t hi,
                                                unsigned long long lim)
{
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((unsigned long long)wadj[mid].y < lim) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// The entry of a big-row list that holds chunk c (the largest cbase <= c).
__device__ __forceinline__ SpBig find_chunk(const SpBig *B, int64_t nb, int64_t c)
{
    int64_t lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if ((int64_t)load_spbig(B, mid).cbase <= c) lo = mid;
        else hi = mid - 1;
    }
    return load_spbig(B, lo);
}

// Warp-collective: the lanes with `want` append v to the far list of `epoch`.
__device__ __forceinline__ void push_far(const SpArgs &a, unsigned epoch, bool want, int32_t v)
{
    const unsigned m = __ballot_sync(kFull, want);
    if (!m) return;
    const unsigned lane = lane_id();
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if ((int)lane == leader) base = atomicAdd(&a.hdr->farcnt[epoch & 1], (unsigned long long)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (!want) return;
    const int64_t pos = (int64_t)base + __popc(m & lanemask_lt());
    if (pos < a.n) a.fq[(int64_t)(epoch & 1) * a.n + pos] = v;
    else record_error(a.st, GB_ERR_RANGE, SITE_SP_FAR, pos);
}

// Warp-collective relaxation of one edge per lane whose distance test has
// been made: dist(v) lowered to nd if still smaller; a lowered v is queued
// near (nd < T) or listed far.
__device__ __forceinline__ void relax_tail(const SpArgs &a, bool cand, int32_t u, int32_t v,
                                           unsigned long long nd, unsigned long long T, unsigned qnext,
                                           unsigned epoch, unsigned long long &won)
{
    bool to_near = false, to_far = false;
    if (cand) {
        const unsigned long long old = atomicMin(&a.dist[v], nd);
        if (nd < old) {
            ++won;
            a.parent[v] = u;
            if (nd < T) to_near = atomicExch(&a.nstamp[v], qnext) != qnext;
            else to_far = atomicExch(&a.fstamp[v], epoch) != epoch;
        }
    }
    push_near(a, qnext, to_near, v);
    push_far(a, epoch, to_far, v);
}

// Two edges per lane: both endpoint distances are read before either atomic,
// so that a warp keeps twice the random reads in flight.
__device__ __forceinline__ void relax2(const SpArgs &a, bool ok0, int32_t u0, uint2 c0,
                                       unsigned long long d0, bool ok1, int32_t u1, uint2 c1,
                                       unsigned long long d1, unsigned long long T, unsigned qnext,
                                       unsigned epoch, unsigned long long &won)
{
    const unsigned long long nd0 = d0 + c0.y, nd1 = d1 + c1.y;
    const unsigned long long cur0 = ok0 ? __ldcg(&a.dist[c0.x]) : 0ull;
    const unsigned long long cur1 = ok1 ? __ldcg(&a.dist[c1.x]) : 0ull;
    relax_tail(a, ok0 && nd0 < cur0, u0, (int32_t)c0.x, nd0, T, qnext, epoch, won);
    relax_tail(a, ok1 && nd1 < cur1, u1, (int32_t)c1.x, nd1, T, qnext, epoch, won);
}

// The row of stream slot k of a warp's 32-row edge stream (the lane whose
// exclusive prefix is the largest <= k).
__device__ __forceinline__ int stream_owner(int64_t excl, int64_t k)
{
    int owner = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        const int cand = owner + step;
        if (__shfl_sync(kFull, excl, cand) <= k) owner = cand;
    }
    return owner;
}

// Warp-collective: relax the edges [so + (k - eo)] of a 32-row stream of
// `total` slots (row starts s0, exclusive prefixes excl, distances du, ids u),
// two slots per lane per step.
__device__ __forceinline__ void relax_stream(const SpArgs &a, uint64_t pol, int64_t total, int64_t s0,
                                             int64_t excl, unsigned long long du, int32_t u,
                                             unsigned long long T, unsigned qnext, unsigned epoch,
                                             unsigned long long &won)
{
    const unsigned lane = lane_id();
    for (int64_t b = 0; b < total; b += 64) {
        const int64_t k0 = b + lane, k1 = b + 32 + lane;
        const int o0 = stream_owner(excl, k0), o1 = stream_owner(excl, k1);
        const int64_t so0 = __shfl_sync(kFull, s0, o0), eo0 = __shfl_sync(kFull, excl, o0);
        const int64_t so1 = __shfl_sync(kFull, s0, o1), eo1 = __shfl_sync(kFull, excl, o1);
        const unsigned long long du0 = __shfl_sync(kFull, du, o0), du1 = __shfl_sync(kFull, du, o1);
        const int32_t u0 = __shfl_sync(kFull, u, o0), u1 = __shfl_sync(kFull, u, o1);
        const bool ok0 = k0 < total, ok1 = k1 < total;
        uint2 c0 = make_uint2(0u, 0u), c1 = make_uint2(0u, 0u);
        if (ok0) c0 = ld_stream(a.wadj + so0 + (k0 - eo0), pol);
        if (ok1) c1 = ld_stream(a.wadj + so1 + (k1 - eo1), pol);
        relax2(a, ok0, u0, c0, du0, ok1, u1, c1, du1, T, qnext, epoch, won);
    }
}

__global__ void __launch_bounds__(SP_THREADS, SP_MINB) sssp_kernel(SpArgs a)
{
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    const unsigned lane = lane_id();
    const int64_t gwarp = gtid >> 5;
    const int64_t nwarps = gthreads >> 5;
    const int64_t n = a.n;
    SpHeader *h = a.hdr;
    unsigned bar = grid_barrier_base(&h->bar);
    unsigned long long processed = 0, scanned = 0, won = 0, reached = 0;
    const uint64_t t_start = globaltimer_ns();
    const uint64_t pol = stream_policy();

    // ---- init: every distance infinite but the root's; the root queued
    for (int64_t v = gtid; v < n; v += gthreads) {
        a.dist[v] = v == a.root ? 0ull : SP_INF;
        a.parent[v] = v == a.root ? a.root : -1;
        a.nstamp[v] = v == a.root ? 1u : 0u;
        a.fstamp[v] = 0u;
        a.sstamp[v] = 0u;
    }
    if (gtid == 0) {
        a.nq[n + 0] = a.root;  // queue 1 sits in slot 1
        h->q[1].cnt = 1;
        h->minfar = SP_INF;
        const int64_t d = a.off[a.root + 1] - a.off[a.root];
        if (d > SP_BIG) {
            h->q[1].big = (1ull << 32) | (unsigned long long)((d + SP_CHUNK - 1) / SP_CHUNK);
            reinterpret_cast<unsigned long long *>(a.bq)[a.bigcap] = (unsigned long long)(uint32_t)a.root;
        }
    }
    if (!grid_sync(&h->bar, bar, a.st, a.timeout_ns, SITE_SP_BAR)) return;

    unsigned qcur = 1, epoch = 1;
    unsigned long long T = a.delta;
    long long rounds = 0, buckets = 0;
    // device time per phase, as thread 0 sees it from barrier to barrier
    unsigned long long ph[4] = {0, 0, 0, 0};
    uint64_t t_ph = globaltimer_ns();
    auto phase_end = [&](int k) {
        if (gtid == 0) {
            const uint64_t now = globaltimer_ns();
            ph[k] += now - t_ph;
            t_ph = now;
        }
    };
    for (;; ++rounds) {
        if (rounds > a.max_rounds) {  // cannot happen: every queued vertex had its distance lowered
            if (gtid == 0) record_error(a.st, GB_ERR_TIMEOUT, SITE_SP_ROUNDS, rounds);
            return;
        }
        // a bound on the whole search: the error makes every block leave at its next barrier
        if (gtid == 0 && globaltimer_ns() - t_start > a.run_limit_ns)
            record_error(a.st, GB_ERR_TIMEOUT, SITE_SP_ROUNDS, rounds);
        const unsigned qnext = qcur + 1;
        // the counters of queue qcur+2; their last readers finished two barriers ago
        if (gtid == 0) {
            h->q[(qcur + 2) & 3].cnt = 0;
            h->q[(qcur + 2) & 3].big = 0;
        }
        const int64_t ncur = (int64_t)__ldcg(&h->q[qcur & 3].cnt);
        const unsigned long long bigc = __ldcg(&h->q[qcur & 3].big);
        const int32_t *Q = a.nq + (int64_t)(qcur & 1) * n;
        // ---- light edges of big rows: chunk c of the queue's numbering, one per warp;
        // an edge is light while w < T - dist(u), a prefix of the weight-sorted row
        const int64_t nb = (int64_t)(bigc >> 32) < a.bigcap ? (int64_t)(bigc >> 32) : a.bigcap;
        const int64_t nch = nb > 0 ? (int64_t)(bigc & 0xffffffffull) : 0;
        const SpBig *B = a.bq + (int64_t)(qcur & 1) * a.bigcap;
        for (int64_t c = gwarp; c < nch; c += nwarps) {
            const SpBig be = find_chunk(B, nb, c);
            const int64_t rs = a.off[be.u], re = a.off[be.u + 1];
            const int64_t s0 = rs + (c - (int64_t)be.cbase) * SP_CHUNK;
            const int64_t e0 = s0 + SP_CHUNK < re ? s0 + SP_CHUNK : re;
            const unsigned long long du = __ldcg(&a.dist[be.u]);
            const unsigned long long lim = T - du;
            if ((unsigned long long)a.wadj[s0].y >= lim) continue;  // the chunk is all heavy
            for (int64_t j0 = s0; j0 < e0; j0 += 64) {
                const int64_t j = j0 + lane;
                uint2 c0 = make_uint2(0u, 0u), c1 = make_uint2(0u, 0u);
                if (j < e0) c0 = ld_stream(a.wadj + j, pol);
                if (j + 32 < e0) c1 = ld_stream(a.wadj + j + 32, pol);
                const bool ok0 = j < e0 && (unsigned long long)c0.y < lim;
                const bool ok1 = j + 32 < e0 && (unsigned long long)c1.y < lim;
                scanned += ok0 + ok1;
                relax2(a, ok0, be.u, c0, du, ok1, be.u, c1, du, T, qnext, epoch, won);
                if (!__any_sync(kFull, ok1)) break;  // past the split
            }
        }
        // ---- every queue entry: listed for its bucket's settle step once; the
        // light prefix of a shorter row expanded, 32 rows per warp as one stream
        for (int64_t i0 = gwarp * 32; i0 < ncur; i0 += nwarps * 32) {
            const int64_t i = i0 + lane;
            int64_t s0 = 0, d = 0, deg = 0;
            unsigned long long du = 0;
            bool first = false;
            int32_t u = 0;
            if (i < ncur) {
                u = __ldcg(&Q[i]);
                s0 = a.off[u];
                deg = a.off[u + 1] - s0;
                du = __ldcg(&a.dist[u]);
                first = atomicExch(&a.sstamp[u], epoch) != epoch;
                d = deg > SP_BIG ? 0 : weight_split(a.wadj, s0, s0 + deg, T - du) - s0;
                ++processed;
                scanned += (unsigned long long)d;
            }
            push_settle(a, first, u, deg);
            const int64_t incl = warp_inclusive_scan(d);
            const int64_t total = __shfl_sync(kFull, incl, 31);
            relax_stream(a, pol, total, s0, incl - d, du, u, T, qnext, epoch, won);
        }
        if (!grid_sync(&h->bar, bar, a.st, a.timeout_ns, SITE_SP_BAR)) return;
        phase_end(0);
        if (__ldcg(&h->q[qnext & 3].cnt) > 0) {
            qcur = qnext;
            continue;
        }
        // ---- the bucket below T is settled: the heavy edges of its vertices,
        // from their final distances (every candidate is >= T: far)
        const unsigned e = epoch;
        if (gtid == 0) h->farcnt[(e + 1) & 1] = 0;  // its last reader was the previous split
        {
            const int64_t ns = (int64_t)__ldcg(&h->settle.cnt);
            const unsigned long long sbig = __ldcg(&h->settle.big);
            const int64_t snb = (int64_t)(sbig >> 32) < a.bigcap ? (int64_t)(sbig >> 32) : a.bigcap;
            const int64_t snch = snb > 0 ? (int64_t)(sbig & 0xffffffffull) : 0;
            const SpBig *SB = a.bq + 2 * a.bigcap;
            for (int64_t c = gwarp; c < snch; c += nwarps) {
                const SpBig be = find_chunk(SB, snb, c);
                const int64_t rs = a.off[be.u], re = a.off[be.u + 1];
                const int64_t s0 = rs + (c - (int64_t)be.cbase) * SP_CHUNK;
                const int64_t e0 = s0 + SP_CHUNK < re ? s0 + SP_CHUNK : re;
                const unsigned long long du = __ldcg(&a.dist[be.u]);
                const unsigned long long lim = T - du;
                if ((unsigned long long)a.wadj[e0 - 1].y < lim) continue;  // the chunk is all light
                for (int64_t j0 = s0; j0 < e0; j0 += 64) {
                    const int64_t j = j0 + lane;
                    uint2 c0 = make_uint2(0u, 0u), c1 = make_uint2(0u, 0u);
                    if (j < e0) c0 = ld_stream(a.wadj + j, pol);
                    if (j + 32 < e0) c1 = ld_stream(a.wadj + j + 32, pol);
                    const bool ok0 = j < e0 && (unsigned long long)c0.y >= lim;
                    const bool ok1 = j + 32 < e0 && (unsigned long long)c1.y >= lim;
                    scanned += ok0 + ok1;
                    relax2(a, ok0, be.u, c0, du, ok1, be.u, c1, du, T, qnext, e, won);
                }
            }
            for (int64_t i0 = gwarp * 32; i0 < ns; i0 += nwarps * 32) {
                const int64_t i = i0 + lane;
                int64_t s0 = 0, d = 0;
                unsigned long long du = 0;
                int32_t u = 0;
                if (i < ns) {
                    u = __ldcg(&a.sq[i]);
                    const int64_t rs = a.off[u], deg = a.off[u + 1] - rs;
                    du = __ldcg(&a.dist[u]);
                    if (deg <= SP_BIG) {
                        s0 = weight_split(a.wadj, rs, rs + deg, T - du);
                        d = rs + deg - s0;
                        scanned += (unsigned long long)d;
                    }
                }
                const int64_t incl = warp_inclusive_scan(d);
                const int64_t total = __shfl_sync(kFull, incl, 31);
                relax_stream(a, pol, total, s0, incl - d, du, u, T, qnext, e, won);
            }
        }
        if (!grid_sync(&h->bar, bar, a.st, a.timeout_ns, SITE_SP_BAR)) return;
        phase_end(1);
        // ---- the least far distance >= T
        if (gtid == 0) {  // every block read the settle list before the barrier above
            h->settle.cnt = 0;
            h->settle.big = 0;
        }
        const int64_t nf = (int64_t)__ldcg(&h->farcnt[e & 1]);
        const int32_t *F = a.fq + (int64_t)(e & 1) * n;
        unsigned long long mn = SP_INF;
        for (int64_t i = gtid; i < nf; i += gthreads) {
            const unsigned long long d = __ldcg(&a.dist[__ldcg(&F[i])]);
            if (d >= T && d < mn) mn = d;
        }
        for (int o = 16; o >= 1; o >>= 1) {
            const unsigned long long x = __shfl_xor_sync(kFull, mn, o);
            mn = x < mn ? x : mn;
        }
        if (lane == 0 && mn != SP_INF) atomicMin(&h->minfar, mn);
        if (!grid_sync(&h->bar, bar, a.st, a.timeout_ns, SITE_SP_BAR)) return;
        phase_end(2);
        const unsigned long long mf = __ldcg(&h->minfar);
        if (mf == SP_INF) break;  // nothing left to settle
        const unsigned long long Tn = (mf / a.delta + 1) * a.delta;
        // ---- split the far list: the new bucket's vertices near, the rest far
        for (int64_t i0 = gwarp * 32; i0 < nf; i0 += nwarps * 32) {
            const int64_t i = i0 + lane;
            int32_t v = 0;
            bool to_near = false, to_far = false;
            if (i < nf) {
                v = __ldcg(&F[i]);
                const unsigned long long d = __ldcg(&a.dist[v]);
                // the list holds each vertex once and nothing else pushes now: plain stamps
                if (d >= T && d < Tn) {
                    to_near = true;
                    a.nstamp[v] = qnext;
                } else if (d >= Tn) {
                    to_far = true;
                    a.fstamp[v] = e + 1;
                }
            }
            push_near(a, qnext, to_near, v);
            push_far(a, e + 1, to_far, v);
        }
        if (!grid_sync(&h->bar, bar, a.st, a.timeout_ns, SITE_SP_BAR)) return;
        phase_end(3);
        if (gtid == 0) h->minfar = SP_INF;  // every block read it before the barrier above
        ++buckets;
        T = Tn;
        epoch = e + 1;
        qcur = qnext;
    }

    // ---- outputs: distances as doubles, the canonical tree
    for (int64_t v0 = gwarp * 32; v0 < n; v0 += nwarps * 32) {
        const int64_t v = v0 + lane;
        unsigned long long dv = SP_INF;
        int64_t rs = 0, d = 0;
        int32_t p = -1;
        bool scan = false;
        if (v < n) {
            dv = __ldcg(&a.dist[v]);
            a.dist_out[v] = dv == SP_INF ? (double)INFINITY : (double)dv * kUnit;
            if (v == a.root) p = a.root;
            if (dv != SP_INF) ++reached;
            if (dv != SP_INF && v != a.root) {
                rs = a.off[v];
                d = a.off[v + 1] - rs;
                scan = true;
                if (!a.canonical) {  // keep the recorded parent if it is tight
                    const int32_t q = __ldcg(&a.parent[v]);
                    if (q >= 0 && (int64_t)q < n) {
                        const int64_t j = find_in_row(a.col, rs, rs + d, q);
                        const unsigned long long dq = __ldcg(&a.dist[q]);
                        if (j >= 0 && dq != SP_INF && dq + a.wgt[j] == dv) {
                            p = q;
                            scan = false;
                        }
                    }
                }
            }
        }
        // short rows: the lane scans its own row in order
        if (scan && d <= 32) {
            for (int64_t j = rs; j < rs + d; ++j) {
                const int32_t u = a.col[j];
                const unsigned long long du = __ldcg(&a.dist[u]);
                if (du != SP_INF && du + a.wgt[j] == dv) {
                    p = u;
                    break;
                }
            }
        }
        // long rows: the warp scans each in rounds of 32 entries
        unsigned longm = __ballot_sync(kFull, scan && d > 32);
        while (longm) {
            const int src = __ffs(longm) - 1;
            longm &= longm - 1;
            const int64_t lrs = __shfl_sync(kFull, rs, src);
            const int64_t ld = __shfl_sync(kFull, d, src);
            const unsigned long long ldv = __shfl_sync(kFull, dv, src);
            int32_t found = -1;
            for (int64_t j0 = lrs; j0 < lrs + ld; j0 += 32) {
                const int64_t j = j0 + lane;
                bool tight = false;
                int32_t u = 0;
                if (j < lrs + ld) {
                    u = a.col[j];
                    const unsigned long long du = __ldcg(&a.dist[u]);
                    tight = du != SP_INF && du + a.wgt[j] == ldv;
                }
                const unsigned tm = __ballot_sync(kFull, tight);
                if (tm) {
                    found = __shfl_sync(kFull, u, __ffs(tm) - 1);
                    break;
                }
            }
            if ((int)lane == src) p = found;
        }
        if (v < n) a.parent[v] = p;
    }
    processed = warp_sum(processed);
    scanned = warp_sum(scanned);
    won = warp_sum(won);
    reached = warp_sum(reached);
    if (lane == 0) {
        atomicAdd(&h->acc[0], processed);
        atomicAdd(&h->acc[1], scanned);
        atomicAdd(&h->acc[2], won);
        atomicAdd(&h->acc[3], reached);
    }
    if (!grid_sync(&h->bar, bar, a.st, a.timeout_ns, SITE_SP_BAR)) return;
    if (gtid == 0 && a.stats) {
        a.stats->rounds = (unsigned long long)rounds + 1;
        a.stats->buckets = (unsigned long long)buckets + 1;
        a.stats->processed = __ldcg(&h->acc[0]);
        a.stats->scanned = __ldcg(&h->acc[1]);
        a.stats->won = __ldcg(&h->acc[2]);
        a.stats->reached = __ldcg(&h->acc[3]);
        a.stats->delta = a.delta;
        for (int k = 0; k < 4; ++k) a.stats->phase_ns[k] = ph[k];
    }
}

// ---------------------------------------------------------------------------
// Validation (the SSSP rules of the Graph500 benchmark; see sssp_validate)
// ---------------------------------------------------------------------------

constexpr int SV_THREADS = 256;
constexpr int SV_TILE = 32 * 64;
constexpr unsigned long long kNoFail = ~0ull;

struct SvAcc {
    unsigned long long first7;   // vertex pass: rule 7
    unsigned long long first2;   // vertex pass: rule 2
    unsigned long long first34;  // parent pass: rules 3, 4
    unsigned long long first56;  // CSR entry pass: rules 5, 6
    unsigned long long reached;
    unsigned long long deg_sum;
    unsigned long long teps;
    unsigned long long max_dist_bits;  // bits of the largest finite distance (>= 0)
    int root_bad;
};

__device__ __forceinline__ void fold_min(unsigned long long f, unsigned long long *dst)
{
    for (int o = 16; o >= 1; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(kFull, f, o);
        f = x < f ? x : f;
    }
    if ((threadIdx.x & 31) == 0 && f != kNoFail) atomicMin(dst, f);
}

__global__ void sv_init_kernel(SvAcc *acc)
{
    acc->first7 = acc->first2 = acc->first34 = acc->first56 = kNoFail;
    acc->reached = acc->deg_sum = acc->teps = acc->max_dist_bits = 0;
    acc->root_bad = 0;
}

__global__ void __launch_bounds__(SV_THREADS) sv_vertex_kernel(const int64_t *__restrict__ off,
                                                               int64_t n, int64_t root,
                                                               const int32_t *__restrict__ parent,
                                                               const double *__restrict__ dist,
                                                               SvAcc *acc)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long f7 = kNoFail, f2 = kNoFail, reached = 0, deg = 0, maxb = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int32_t p = parent[v];
        const double d = dist[v];
        if (v == root && (p != root || d != 0.0)) acc->root_bad = 1;
        if (p < -1 || (int64_t)p >= n || isnan(d) || d < 0.0) {
            if (f7 == kNoFail) f7 = ((unsigned long long)v << 3) | 7u;
        } else if ((p == -1) != (isinf(d) != 0)) {
            if (f2 == kNoFail) f2 = ((unsigned long long)v << 3) | 2u;
        }
        if (!isinf(d) && !isnan(d) && d >= 0.0) {
            ++reached;
            deg += (unsigned long long)(off[v + 1] - off[v]);
            const unsigned long long b = (unsigned long long)__double_as_longlong(d);
            maxb = b > maxb ? b : maxb;  // non-negative doubles order as their bits
        }
    }
    fold_min(f7, &acc->first7);
    fold_min(f2, &acc->first2);
    reached = warp_sum(reached);
    deg = warp_sum(deg);
    for (int o = 16; o >= 1; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(kFull, maxb, o);
        maxb = x > maxb ? x : maxb;
    }
    if ((threadIdx.x & 31) == 0) {
        if (reached) atomicAdd(&acc->reached, reached);
        if (deg) atomicAdd(&acc->deg_sum, deg);
        if (maxb) atomicMax(&acc->max_dist_bits, maxb);
    }
}

// Rules 3, 4: the parent is found in v's sorted row by bisection.
__global__ void __launch_bounds__(SV_THREADS) sv_parent_kernel(const int64_t *__restrict__ off,
                                                               const int32_t *__restrict__ col,
                                                               const uint32_t *__restrict__ wgt,
                                                               int64_t n, int64_t root,
                                                               const int32_t *__restrict__ parent,
                                                               const double *__restrict__ dist,
                                                               SvAcc *acc)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long first = kNoFail;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n && first == kNoFail;
         v += stride) {
        const int32_t p = parent[v];
        const double d = dist[v];
        if (v == root || p < 0 || (int64_t)p >= n || isinf(d) || isnan(d) || d < 0.0) continue;
        const int64_t j = find_in_row(col, off[v], off[v + 1], p);
        unsigned code = 0;
        if (j < 0) code = 3;
        else if (dist[p] + (double)wgt[j] * kUnit != d) code = 4;
        if (code) first = ((unsigned long long)v << 3) | code;
    }
    fold_min(first, &acc->first34);
}

// Rules 5, 6 over every CSR entry (u, col[e]): a warp takes SV_TILE entries,
// each lane finds the row of its first entry by bisection and walks forward.
__global__ void __launch_bounds__(SV_THREADS) sv_edge_kernel(const int64_t *__restrict__ off,
                                                             const int32_t *__restrict__ col,
                                                             const uint32_t *__restrict__ wgt,
                                                             int64_t n, int64_t nnz,
                                                             const double *__restrict__ dist,
                                                             SvAcc *acc)
{
    const unsigned lane = threadIdx.x & 31u;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long first = kNoFail;
    for (int64_t e0 = gwarp * SV_TILE; e0 < nnz; e0 += nwarps * SV_TILE) {
        int64_t e = e0 + lane;
        if (e >= nnz) continue;
        int64_t lo = 0, hi = n;  // largest u with off[u] <= e
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (off[mid] <= e) lo = mid;
            else hi = mid;
        }
        int64_t u = lo;
        const int64_t e_end = e0 + SV_TILE < nnz ? e0 + SV_TILE : nnz;
        for (; e < e_end && first == kNoFail; e += 32) {
            while (off[u + 1] <= e) ++u;
            const int32_t v = col[e];
            if (v < 0 || (int64_t)v >= n) continue;
            const double du = dist[u], dv = dist[v];
            unsigned code = 0;
            if ((isinf(du) != 0) != (isinf(dv) != 0)) code = 5;
            else if (!isinf(du) && dv > du + (double)wgt[e] * kUnit) code = 6;
            if (code) first = ((unsigned long long)e << 3) | code;
        }
    }
    fold_min(first, &acc->first56);
}

__global__ void __launch_bounds__(SV_THREADS) sv_teps_kernel(const int64_t *__restrict__ start,
                                                             int64_t m, int64_t n,
                                                             const double *__restrict__ dist,
                                                             SvAcc *acc)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long cnt = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int64_t u = start[e];
        if (u >= 0 && u < n && !isinf(dist[u])) ++cnt;
    }
    cnt = warp_sum(cnt);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&acc->teps, cnt);
}

int sssp_pick_blocks(int num_sms)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sssp_kernel, SP_THREADS, 0) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    return num_sms * std::min(per_sm, SP_MINB);
}

}  // namespace

gb_status build_csr_weighted(const int64_t *edges, const float *w, int64_t m, int scale, gb_graph *g,
                             cudaStream_t s)
{
    gb_status rc = build_csr(edges, m, scale, g, s);
    if (rc != GB_OK) return rc;
    Context *ctx = context();
    GB_CUDA(gb::dmalloc(&g->wgt, std::max<int64_t>(g->nnz, 4) * sizeof(uint32_t)));
    GB_CUDA(cudaMemsetAsync(g->wgt, 0xff, std::max<int64_t>(g->nnz, 4) * sizeof(uint32_t), s));
    if (m > 0) {
        wt_attach_kernel<<<ctx->num_sms * 8, 256, 0, s>>>(edges, w, m, g->off, g->col, g->n, g->wgt,
                                                          ctx->status);
        note_launch();
        GB_CUDA(cudaGetLastError());
    }
    DevStatus hst;
    GB_CUDA(cudaMemcpyAsync(&hst, ctx->status, sizeof(hst), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    if (hst.code != 0) {
        GB_CUDA(cudaMemsetAsync(ctx->status, 0, sizeof(DevStatus), s));
        GB_CUDA(cudaStreamSynchronize(s));
        set_error(hst.where == SITE_SP_W ? "graph_build_csr_weighted: a weight outside (0, 1]"
                                         : "graph_build_csr_weighted: device error while attaching weights");
        return (gb_status)hst.code;
    }
    // the rows by ascending weight: one sort of (row << 25 | weight) keys with the columns
    const int64_t nnz = g->nnz;
    GB_CUDA(gb::dmalloc(&g->wadj, std::max<int64_t>(nnz, 4) * sizeof(uint2)));
    if (nnz > 0) {
        uint64_t *k0 = nullptr, *k1 = nullptr, *ks = nullptr;
        uint32_t *v0 = nullptr, *v1 = nullptr, *vs = nullptr;
        Scratch tmp(s);
        GB_CUDA(tmp.alloc(&k0, (size_t)nnz));
        GB_CUDA(tmp.alloc(&k1, (size_t)nnz));
        GB_CUDA(tmp.alloc(&v0, (size_t)nnz));
        GB_CUDA(tmp.alloc(&v1, (size_t)nnz));
        wsort_keys_kernel<<<ctx->num_sms * 8, 256, 0, s>>>(g->off, g->col, g->wgt, g->n, k0, v0);
        note_launch();
        GB_CUDA(cudaGetLastError());
        gb_status rc2 = radix_sort(k0, k1, v0, v1, nnz, 0, 25 + scale, &ks, &vs, s);
        if (rc2 != GB_OK) return rc2;
        wsort_pack_kernel<<<ctx->num_sms * 8, 256, 0, s>>>(ks, vs, nnz, g->wadj);
        note_launch();
        GB_CUDA(cudaGetLastError());
    }
    GB_CUDA(cudaStreamSynchronize(s));
    return GB_OK;
}

gb_status sssp_impl(const gb_graph *g, int64_t root, double delta, double *dist, int32_t *parent,
                    SsspDevStats *stats, cudaStream_t s)
{
    Context *ctx = context();
    if (!ctx) return GB_ERR_CUDA;
    if (!g->wgt || !g->wadj) {
        set_error("sssp: the graph has no weights (build it with graph_build_csr_weighted)");
        return GB_ERR_INVALID;
    }
    const int64_t n = g->n;
    const int64_t bigcap = g->nnz / SP_BIG + 2;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    // header | dist | near, far and settle stamps | near queues | far lists |
    // settle list | big lists (2 near slots, then the settle list's); slot k of
    // a region at base + k * size
    const size_t o_dist = al(sizeof(SpHeader));
    const size_t o_ns = o_dist + al(8 * (size_t)n);
    const size_t o_fs = o_ns + al(4 * (size_t)n);
    const size_t o_ss = o_fs + al(4 * (size_t)n);
    const size_t o_nq = o_ss + al(4 * (size_t)n);
    const size_t o_fq = o_nq + al(8 * (size_t)n);
    const size_t o_sq = o_fq + al(8 * (size_t)n);
    const size_t o_bq = o_sq + al(4 * (size_t)n);
    const size_t total = o_bq + al(24 * (size_t)bigcap);
    unsigned char *ws = nullptr;
    Scratch tmp(s);
    GB_CUDA(tmp.alloc(&ws, total));
    GB_CUDA(cudaMemsetAsync(ws, 0, sizeof(SpHeader), s));
    SpArgs a;
    a.off = g->off;
    a.col = g->col;
    a.wgt = g->wgt;
    a.wadj = g->wadj;
    a.n = n;
    a.root = (int32_t)root;
    a.dist = reinterpret_cast<unsigned long long *>(ws + o_dist);
    a.nstamp = reinterpret_cast<uint32_t *>(ws + o_ns);
    a.fstamp = reinterpret_cast<uint32_t *>(ws + o_fs);
    a.sstamp = reinterpret_cast<uint32_t *>(ws + o_ss);
    a.nq = reinterpret_cast<int32_t *>(ws + o_nq);
    a.fq = reinterpret_cast<int32_t *>(ws + o_fq);
    a.sq = reinterpret_cast<int32_t *>(ws + o_sq);
    a.bq = reinterpret_cast<SpBig *>(ws + o_bq);
    a.bigcap = bigcap;
    a.hdr = reinterpret_cast<SpHeader *>(ws);
    a.st = ctx->status;
    a.stats = stats;
    const double du = std::floor(delta * 16777216.0 + 0.5);
    a.delta = (unsigned long long)std::max(1.0, std::min(du, 4.0e18));
    a.dist_out = dist;
    a.parent = parent;
    a.canonical = options().canonical_parents;
    a.timeout_ns = timeout_ns();
    a.run_limit_ns = 8 * a.timeout_ns;
    a.max_rounds = (long long)1 << 31;  // round ids are 32-bit stamps
    static int blocks_cache[64] = {0};
    const int dev = ctx->device;
    int blocks = dev < 64 ? blocks_cache[dev] : 0;
    if (blocks == 0) {
        blocks = sssp_pick_blocks(ctx->num_sms);
        if (dev < 64) blocks_cache[dev] = blocks;
    }
    void *args[] = {&a};
    GB_CUDA(cudaLaunchCooperativeKernel((const void *)sssp_kernel, dim3(blocks), dim3(SP_THREADS), args,
                                        0, s));
    note_launch();
    return GB_OK;
}

gb_status sssp_validate_impl(const gb_graph *g, int64_t root, const int32_t *parent, const double *dist,
                             const int64_t *edges, int64_t m, gb_sssp_validation *out, cudaStream_t s)
{
    Context *ctx = context();
    if (!ctx) return GB_ERR_CUDA;
    if (!g->wgt) {
        set_error("sssp_validate: the graph has no weights");
        return GB_ERR_INVALID;
    }
    gb_sssp_validation r;
    r.code = 0;
    r.pad = 0;
    r.where = -1;
    r.reached = 0;
    r.component_edges = 0;
    r.teps_edges = edges ? 0 : -1;
    r.max_dist = 0.0;
    if (root < 0 || root >= g->n) {
        r.code = 7;
        r.where = root;
        *out = r;
        return GB_OK;
    }
    SvAcc *acc = nullptr;
    Scratch tmp(s);
    GB_CUDA(tmp.alloc(&acc, 1));
    const int grid = ctx->num_sms * 8;
    sv_init_kernel<<<1, 1, 0, s>>>(acc);
    note_launch();
    sv_vertex_kernel<<<grid, SV_THREADS, 0, s>>>(g->off, g->n, root, parent, dist, acc);
    note_launch();
    sv_parent_kernel<<<grid, SV_THREADS, 0, s>>>(g->off, g->col, g->wgt, g->n, root, parent, dist, acc);
    note_launch();
    if (g->nnz > 0) {
        sv_edge_kernel<<<grid, SV_THREADS, 0, s>>>(g->off, g->col, g->wgt, g->n, g->nnz, dist, acc);
        note_launch();
    }
    if (edges && m > 0) {
        sv_teps_kernel<<<grid, SV_THREADS, 0, s>>>(edges, m, g->n, dist, acc);
        note_launch();
    }
    GB_CUDA(cudaGetLastError());
    SvAcc h;
    GB_CUDA(cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
    GB_CUDA(tmp.drop(acc));
    GB_CUDA(cudaStreamSynchronize(s));
    r.reached = (int64_t)h.reached;
    r.component_edges = (int64_t)(h.deg_sum / 2);
    if (edges) r.teps_edges = (int64_t)h.teps;
    double md = 0.0;
    std::memcpy(&md, &h.max_dist_bits, sizeof(md));
    r.max_dist = md;
    // the serial order: the range pass, rule 1, rule 2, the parents, the CSR entries
    auto take = [&](unsigned long long f) {
        if (r.code == 0 && f != kNoFail) {
            r.code = (int32_t)(f & 7ull);
            r.where = (int64_t)(f >> 3);
        }
    };
    take(h.first7);
    if (r.code == 0 && h.root_bad) {
        r.code = 1;
        r.where = root;
    }
    take(h.first2);
    take(h.first34);
    take(h.first56);
    *out = r;
    return GB_OK;
}

}  // namespace gb
