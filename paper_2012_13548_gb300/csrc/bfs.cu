// Kernel 2 (Sec. 2.3): level-synchronous, direction-optimising BFS.
//
// One persistent cooperative kernel runs the whole search; levels are
// separated by a software grid barrier (bounded waits), which is the level
// synchronisation of Sec. 2.3.2 (all vertices of a level are handled together
// and the next level starts only once the whole level is done; the section
// also shows the wrong levels a search gets without it).  Per level the kernel runs one
// of two steps, chosen identically by every block from global counters:
//
//  top-down (Algorithm "Parallel BFS", Sec. 2.3.2): for every frontier vertex
//    and every neighbour in parallel, an unvisited neighbour is claimed with
//    an atomic OR on the visited bitmap; the winner records parent and level
//    and appends the vertex to the next queue with one atomic per warp.
//    Frontier vertices of degree <= big_degree are expanded 32 at a time by a
//    warp that gathers their adjacency lists as one contiguous stream of
//    edges; larger ones are cut into 128-edge chunks spread over all warps.
//  bottom-up (Beamer, Asanovic, Patterson, SC 2012): every unvisited vertex
//    scans its sorted adjacency list and stops at the first neighbour in the
//    frontier bitmap, which is therefore the smallest-id parent.  Outside
//    canonical mode it first tests its hub (a neighbour of largest degree,
//    built with the graph): a hub in the frontier is a valid parent, found
//    without reading the row, and a row of one entry whose hub is not in the
//    frontier is settled without reading it either.
//
// The switch follows Beamer: top-down -> bottom-up when the frontier's edges
// exceed (edges of unvisited vertices) / alpha, back when the frontier is
// shrinking and smaller than n / beta.  Both steps leave the next frontier as
// a queue and as a bitmap, so switching costs nothing.  In canonical mode the
// parents of vertices claimed top-down are recomputed at the next level as
// their smallest-id neighbour in the previous frontier, which makes the tree
// the unique one the oracle derives from the level array (Sec. 2.3.1).
//
// Memory layout of one search: visited bitmap and a ring of four frontier
// bitmaps (n/8 bytes each, L2-resident at SCALE 26: 8 MB), one int32 queue of
// n entries holding every level's frontier back to back (the BFS order), one
// state byte per vertex (level and parent source, mostly L2-resident: 64 MB at
// SCALE 26), a list of big frontier vertices with their chunk bases, and four
// level control records (ring).  The level and parent outputs are written once,
// by a last pass over all vertices.
#include "common.cuh"
#include "internal.h"

#include <algorithm>
#include <mutex>
#include <string>

namespace gb {
namespace {

constexpr int BFS_THREADS = 512;
constexpr int BIG_CHUNK = 128;      // edges per chunk of a big frontier vertex (one round)
constexpr int BU_LANE_FIRST = 8;    // bottom-up: each lane probes this many neighbours itself
constexpr int BU_WORDS = 2;         // bottom-up hub pass: visited words (or 32-entry list groups) per warp step
constexpr int PBUF = 256;           // per-warp ring of vertices left for the row pass
constexpr int BFS_WARPS = BFS_THREADS / 32;
constexpr int QBUF = 512;           // per-warp buffer of discovered vertices (shared memory)
constexpr int BBUF = 32;            // per-warp buffer of discovered big-degree vertices
constexpr int SITE_BFS_BAR = 20;
constexpr int SITE_BFS_LEVELS = 21;

// With GB_CHECKED defined every global index below is tested first; a bad
// one is recorded in the status word (site, index) and the access skipped.
#ifdef GB_CHECKED
#define GB_OK_IDX(st, i, bound, site) \
    ((int64_t)(i) >= 0 && (int64_t)(i) < (int64_t)(bound) \
         ? true : (record_error((st), GB_ERR_RANGE, (site), (long long)(i)), false))
#else
#define GB_OK_IDX(st, i, bound, site) true
#endif

struct LevelCtl {
    unsigned long long qcnt;  // vertices appended to the next queue
    unsigned long long mf;    // sum of their degrees
    unsigned long long big;   // (count << 32) | chunks of big vertices appended
    unsigned long long pad;
};

struct BigEnt {
    int32_t u;
    uint32_t cbase;
};

struct WsHeader {
    GridBarrier bar;
    unsigned done;
    unsigned pad0;
    LevelCtl ctl[4];
    unsigned long long acc[6];  // edges, touched, reached, nlevels, td, bu
    unsigned long long t0;      // global timer at the end of the init phase
};

struct BfsArgs {
    const int64_t *off;
    const int32_t *col;
    const uint32_t *nz;  // degree >= 1 bitmap
    const int32_t *hub;  // per vertex a neighbour of largest degree (-1: none); null: unused
    int64_t n;
    int64_t nnz;
    int32_t root;
    int32_t *parent;
    int32_t *level;
    uint8_t *st8;  // per vertex: level + 1 (7 bits) and "parent is the hub" (bit 7)
    unsigned *vis;
    unsigned *fb;  // 4 bitmaps of nw words
    int64_t nw;
    int32_t *queue;
    int32_t *ulist;  // per warp a segment of useg entries: the vertices a bottom-up level left open (or null)
    int64_t useg;
    const int32_t *nzl;  // the vertices of degree >= 1, ascending (or null)
    const int2 *hd;         // (hub, min(degree, 65535)) per vertex (set whenever ulist is)
    int64_t nnzv;
    BigEnt *bigq;
    int64_t bigcap;
    WsHeader *hdr;
    DevStatus *st;
    BfsDevStats *stats;
    float alpha;
    float beta;
    int big_deg;
    int canonical;
    int vec_out;  // parent, level, hub and the state bytes allow 16-byte vector access
    int vec_col;  // col is 16-byte aligned and padded to a multiple of 4 entries
    uint64_t timeout_ns;
};

// The big list is written by other blocks during the previous level: read it
// from L2, never from a possibly stale L1 line.
__device__ __forceinline__ BigEnt load_big(const BigEnt *q, int64_t i)
{
    const unsigned long long r = __ldcg(reinterpret_cast<const unsigned long long *>(q) + i);
    BigEnt b;
    b.u = (int32_t)(r & 0xffffffffull);
    b.cbase = (uint32_t)(r >> 32);
    return b;
}

// Chunks of a big vertex start at 16-byte boundaries of the column array
// (the row start rounded down to a multiple of 4 entries, then every
// BIG_CHUNK entries), so that every lane reads its four entries of a chunk
// with one aligned 16-byte load; a row of deg entries spans at most this
// many such chunks (one may come out empty).
__device__ __forceinline__ unsigned nchunks(int64_t deg)
{
    return (unsigned)((deg + 3 + BIG_CHUNK - 1) / BIG_CHUNK);
}

// The outputs are not written level by level: a search would then rewrite
// scattered parts of almost every 32-byte sector of the two n-entry output
// arrays at every large level, each a read-modify-write in DRAM.  A reached
// vertex records one byte instead (its level + 1, and whether its parent is
// its hub, which the bottom-up hub test then need not store), and the last
// pass writes level and parent of every vertex as whole lines.  A parent
// found any other way is written to the parent output at once (few: the
// top-down claims and the row-pass finds).  Levels from ST_ESC - 1 up are
// written to the level output directly and flagged ST_ESC.
constexpr unsigned ST_HUB = 0x80u;
constexpr unsigned ST_ESC = 0x7fu;

__device__ __forceinline__ void mark_reached(const BfsArgs &a, int64_t v, int lvl, bool via_hub)
{
    unsigned e = (unsigned)lvl + 1u;
    if (e >= ST_ESC) {
        e = ST_ESC;
        a.level[v] = lvl;
    }
    a.st8[v] = (uint8_t)(e | (via_hub ? ST_HUB : 0u));
}

// Discovered vertices are staged per warp in shared memory and moved to the
// global queue with one atomic per flush, so that the level counters see a
// few atomics per warp instead of one per 32 discoveries.  The fill levels
// are warp-uniform registers: every lane adds the same ballot counts, so no
// lane ever reads a count another lane is writing.
struct WarpBuf {
    int32_t q[QBUF];
    unsigned long long b[BBUF];  // v | nchunks << 32
    int32_t pu[PBUF];            // bottom-up: vertices waiting for a row pass
};

// Warp-collective: move the staged queue entries to the next level's queue.
__device__ __forceinline__ void flush_queue(WarpBuf &wb, int &qn, const BfsArgs &a,
                                            LevelCtl *nxt, int64_t qnext_base)
{
    if (qn == 0) return;
    __syncwarp();  // the lanes' buffer writes are visible to the whole warp
    const unsigned lane = lane_id();
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&nxt->qcnt, (unsigned long long)qn);
    base = __shfl_sync(kFull, base, 0);
    for (int i = lane; i < qn; i += 32)
        if (GB_OK_IDX(a.st, qnext_base + (int64_t)base + i, a.n, 200))
            __stcg(&a.queue[qnext_base + (int64_t)base + i], wb.q[i]);
    __syncwarp();  // every lane has read the buffer before it is refilled
    qn = 0;
}

// Warp-collective: give the staged big vertices their chunk ranges and list them.
__device__ __forceinline__ void flush_big(WarpBuf &wb, int &bn, const BfsArgs &a, LevelCtl *nxt,
                                          int64_t bnext_base)
{
    if (bn == 0) return;
    __syncwarp();
    const unsigned lane = lane_id();
    const unsigned long long e = (int)lane < bn ? wb.b[lane] : 0ull;
    const unsigned nch = (unsigned)(e >> 32);
    const unsigned incl = warp_inclusive_scan(nch);
    const unsigned total = __shfl_sync(kFull, incl, 31);
    unsigned long long p = 0;
    if (lane == 0) p = atomicAdd(&nxt->big, ((unsigned long long)bn << 32) | total);
    p = __shfl_sync(kFull, p, 0);
    if ((int)lane < bn && GB_OK_IDX(a.st, bnext_base + (int64_t)(p >> 32) + lane, a.bigcap, 202)) {
        const unsigned long long cb = (p & 0xffffffffull) + incl - nch;
        __stcg(reinterpret_cast<unsigned long long *>(a.bigq) + bnext_base + (int64_t)(p >> 32) + lane,
               (e & 0xffffffffull) | (cb << 32));
    }
    __syncwarp();
    bn = 0;
}

// Warp-collective: the lanes with `keep` stay open for the next level.  A
// bottom-up level lists the vertices it leaves open in the warp's own segment
// of the open list (no atomics: the warp owns the segment), and a bottom-up
// level that follows lets the same warp walk that segment instead of its
// words of the visited bitmap, compacting it in place (a vertex is written
// back only after it and every vertex before it were read).
__device__ __forceinline__ void append_open(bool keep, int32_t u, int32_t *seg, int &un)
{
    if (!seg) return;
    const unsigned bal = __ballot_sync(kFull, keep);
    if (keep) __stcg(&seg[un + __popc(bal & lanemask_lt())], u);
    un += __popc(bal);
}

// Warp-collective: set the visited and next-frontier bits of the lanes with
// `on`.  Lanes that hold vertices of the same bitmap word next to each other
// (the lists are in increasing vertex order) form a run; an OR scan within
// the runs gives the last lane of each run the run's bits, and that lane sets
// them with one atomic per bitmap.  Lanes of one word that are not adjacent
// only cost an extra atomic.
__device__ __forceinline__ void set_bits(bool on, int32_t u, unsigned *vis, unsigned *Fn)
{
    const int lane = (int)lane_id();
    const int w = on ? (int)((unsigned)u >> 5) : -1;
    unsigned bits = on ? 1u << (u & 31) : 0u;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned ob = __shfl_up_sync(kFull, bits, d);
        const int ow = __shfl_up_sync(kFull, w, d);
        if (lane >= d && ow == w) bits |= ob;
    }
    const int wnext = __shfl_down_sync(kFull, w, 1);
    if (on && (lane == 31 || wnext != w)) {
        atomicOr(&vis[w], bits);
        atomicOr(&Fn[w], bits);
    }
}

// Warp-collective: the lanes with `won` join the next frontier.
__device__ __forceinline__ void append_next(bool won, int32_t v, int64_t dv, const BfsArgs &a,
                                            WarpBuf &wb, int &qn, int &bn,
                                            unsigned long long &my_mf, LevelCtl *nxt,
                                            int64_t qnext_base, int64_t bnext_base)
{
    const unsigned bal = __ballot_sync(kFull, won);
    if (bal == 0) return;
    const int cnt = __popc(bal);
    if (qn + cnt > QBUF) flush_queue(wb, qn, a, nxt, qnext_base);
    if (won) {
        const int pos = qn + __popc(bal & lanemask_lt());
        if (GB_OK_IDX(a.st, pos, QBUF, 203)) wb.q[pos] = v;
        my_mf += (unsigned long long)dv;
    }
    qn += cnt;
    const bool big = won && dv > a.big_deg;
    const unsigned bb = __ballot_sync(kFull, big);
    if (bb) {
        const int bc = __popc(bb);
        if (bn + bc > BBUF) flush_big(wb, bn, a, nxt, bnext_base);
        if (big) {
            const int pos = bn + __popc(bb & lanemask_lt());
            if (GB_OK_IDX(a.st, pos, BBUF, 204))
                wb.b[pos] = (unsigned long long)(uint32_t)v | ((unsigned long long)nchunks(dv) << 32);
        }
        bn += bc;
    }
}

// Warp-collective top-down visit of TD_E edges per lane (src[t] -> v[t] where
// valid[t]): the visited-bit tests of the TD_E edges are issued together, then
// the claiming atomics together with the candidates' degree loads (a winner
// needs its degree for the next frontier's counters).
constexpr int TD_E = 4;
static_assert(BIG_CHUNK == 32 * TD_E, "a big-vertex chunk is one TD_E-entry group per lane");
__device__ __forceinline__ void td_visit(const bool (&valid)[TD_E], const int32_t (&src)[TD_E],
                                         const int32_t (&v)[TD_E], int l, const BfsArgs &a,
                                         unsigned *Fn, WarpBuf &wb, int &qn, int &bn,
                                         unsigned long long &my_mf, LevelCtl *nxt,
                                         int64_t qnext_base, int64_t bnext_base)
{
    bool cand[TD_E], won[TD_E];
#pragma unroll
    for (int t = 0; t < TD_E; ++t) {
        cand[t] = valid[t] && GB_OK_IDX(a.st, v[t], a.n, 205) &&
                  !((ldcg_u32(&a.vis[(unsigned)v[t] >> 5]) >> (v[t] & 31)) & 1u);
    }
    // the candidates' degrees are loaded with the claims, not after them
    int64_t dv[TD_E];
#pragma unroll
    for (int t = 0; t < TD_E; ++t) dv[t] = cand[t] ? __ldg(&a.off[v[t] + 1]) - __ldg(&a.off[v[t]]) : 0;
#pragma unroll
    for (int t = 0; t < TD_E; ++t) {
        won[t] = false;
        if (cand[t]) {
            const unsigned bit = 1u << (v[t] & 31);
            won[t] = !(atomicOr(&a.vis[(unsigned)v[t] >> 5], bit) & bit);
        }
    }
#pragma unroll
    for (int t = 0; t < TD_E; ++t) {
        if (won[t]) {
            a.parent[v[t]] = src[t];
            mark_reached(a, v[t], l + 1, false);
            atomicOr(&Fn[(unsigned)v[t] >> 5], 1u << (v[t] & 31));
        } else {
            dv[t] = 0;
        }
    }
#pragma unroll
    for (int t = 0; t < TD_E; ++t)
        append_next(won[t], v[t], dv[t], a, wb, qn, bn, my_mf, nxt, qnext_base, bnext_base);
}

// Warp-collective: the row tails [j, e) of the lanes with `open` are scanned
// together.  Each round deals 4 x 32 neighbour slots, an equal share to every
// row still open (consecutive slots of a row are consecutive CSR entries), so
// rows that find their parent leave and the loads of a round are all in
// flight at once.  The first slot of a row whose neighbour is in the frontier
// gives the smallest-id parent.
__device__ __forceinline__ void bu_stream_rows(const BfsArgs &a, const unsigned *F, bool open,
                                               int64_t j, int64_t e, int32_t &found,
                                               unsigned long long &my_edges)
{
    const int lane = (int)lane_id();
    while (true) {
        const bool act = open && found < 0 && j < e;
        const unsigned am = __ballot_sync(kFull, act);
        if (!am) break;
        const int q = 128 / __popc(am);
        const int64_t rem = act ? e - j : 0;
        const int len = (int)(rem < q ? rem : q);
        const int incl = warp_inclusive_scan(len);
        const int total = __shfl_sync(kFull, incl, 31);
        const int excl = incl - len;
        int32_t vv[4];
        unsigned fw[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int k = t * 32 + lane;
            int o = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int c = o + step;
                if (__shfl_sync(kFull, excl, c) <= k) o = c;
            }
            const int64_t jo = __shfl_sync(kFull, j, o);
            const int eo = __shfl_sync(kFull, excl, o);
            const int64_t pos = jo + (k - eo);
            vv[t] = k < total && GB_OK_IDX(a.st, pos, a.nnz, 218) ? __ldg(&a.col[pos]) : -1;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
            fw[t] = vv[t] >= 0 && GB_OK_IDX(a.st, vv[t], a.n, 219) ? ldcg_u32(&F[vv[t] >> 5]) : 0u;
        // each row owner looks for the first hit among its slots, group by group
        int32_t got = -1;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const bool h = vv[t] >= 0 && ((fw[t] >> (vv[t] & 31)) & 1u);
            const unsigned hm = __ballot_sync(kFull, h);
            const int a0 = excl - t * 32, a1 = excl + len - t * 32;
            const int lo = a0 > 0 ? a0 : 0, hi = a1 < 32 ? a1 : 32;
            unsigned seg = 0;
            if (len > 0 && hi > lo) seg = (hi >= 32 ? kFull : ((1u << hi) - 1u)) & ~((1u << lo) - 1u);
            const unsigned mine = hm & seg;
            const int fl = mine ? __ffs(mine) - 1 : 0;
            const int32_t cand = __shfl_sync(kFull, vv[t], fl);
            if (got < 0 && mine) {
                got = cand;
                my_edges += (unsigned long long)(32 * t + fl - excl + 1);
            }
        }
        if (got >= 0) {
            found = got;
        } else {
            my_edges += (unsigned long long)len;
            j += len;
        }
    }
}

// Warp-collective bottom-up row pass over `cnt` (<= 32) vertices of the warp's
// pending ring from position `head`, lane i taking entry head + i: the lane probes the first
// BU_LANE_FIRST neighbours of its row, rows still open are streamed by the
// warp; the first frontier neighbour in row order is the parent.  Entries come
// from several visited words, so the visited and next-frontier bits are set
// with atomics.
__device__ __forceinline__ void bu_row_pass(const BfsArgs &a, const unsigned *F, unsigned *Fn,
                                            int head, int cnt, int l, WarpBuf &wb, int &qn, int &bn,
                                            int32_t *seg, int &un, unsigned long long &my_mf,
                                            unsigned long long &my_edges, LevelCtl *nxt,
                                            int64_t qnext_base, int64_t bnext_base)
{
    const int lane = (int)lane_id();
    __syncwarp();  // the entries, and the commits of their words, are visible to the warp
    const bool act = lane < cnt;
    const int32_t u = act ? wb.pu[(head + lane) & (PBUF - 1)] : 0;
    __syncwarp();  // read before the ring is refilled
    // the offsets were read by this warp in the hub pass: L1 hits
    const int64_t s = act ? __ldg(&a.off[u]) : 0;
    const int32_t d = act ? (int32_t)(__ldg(&a.off[u + 1]) - s) : 0;
    const int32_t la = d < BU_LANE_FIRST ? d : BU_LANE_FIRST;
    int32_t vv[BU_LANE_FIRST];
    unsigned fw[BU_LANE_FIRST];
#pragma unroll
    for (int t = 0; t < BU_LANE_FIRST; ++t)
        vv[t] = t < la && GB_OK_IDX(a.st, s + t, a.nnz, 222) ? __ldg(&a.col[s + t]) : -1;
#pragma unroll
    for (int t = 0; t < BU_LANE_FIRST; ++t)
        fw[t] = vv[t] >= 0 && GB_OK_IDX(a.st, vv[t], a.n, 223) ? ldcg_u32(&F[vv[t] >> 5]) : 0u;
    int hit = -1;
#pragma unroll
    for (int t = 0; t < BU_LANE_FIRST; ++t)
        if (hit < 0 && vv[t] >= 0 && ((fw[t] >> (vv[t] & 31)) & 1u)) hit = t;
    int32_t found = -1;
#pragma unroll
    for (int t = 0; t < BU_LANE_FIRST; ++t)  // select without indexing registers
        if (hit == t) found = vv[t];
    my_edges += (unsigned long long)(hit >= 0 ? hit + 1 : la);
    bu_stream_rows(a, F, act && found < 0 && la < d, s + la, s + d, found, my_edges);
    const bool won = act && found >= 0 && GB_OK_IDX(a.st, u, a.n, 224);
    if (won) {
        a.parent[u] = found;
        mark_reached(a, u, l + 1, false);
        const unsigned bit = 1u << (u & 31);
        atomicOr(&a.vis[(unsigned)u >> 5], bit);
        atomicOr(&Fn[(unsigned)u >> 5], bit);
    }
    append_next(won, u, d, a, wb, qn, bn, my_mf, nxt, qnext_base, bnext_base);
    append_open(act && !won, u, seg, un);  // still no parent: open at the next level
}

// Canonical mode: the vertices claimed top-down at the previous level (queue
// entries [qbase, qbase + qn)) get as parent their smallest-id neighbour in
// that level's frontier Fp, the first one in row order.  32 vertices per warp,
// their rows streamed together, so that a long row (a hub claimed next to the
// root) is scanned by the whole warp rather than by one thread.  Kept out of
// line: the fast path does not carry its code.
__device__ __noinline__ void canonical_rescan(const BfsArgs &a, const unsigned *Fp, int64_t qbase,
                                              int64_t qn, int64_t gwarp, int64_t nwarps)
{
    const int lane = (int)lane_id();
    unsigned long long examined = 0;
    for (int64_t i0 = gwarp * 32; i0 < qn; i0 += nwarps * 32) {
        const int64_t i = i0 + lane;
        int32_t u = 0;
        int64_t s = 0, e = 0;
        if (i < qn && GB_OK_IDX(a.st, qbase + i, a.n, 226)) {
            u = ldcg_i32(&a.queue[qbase + i]);
            if (GB_OK_IDX(a.st, u, a.n, 227)) {
                s = a.off[u];
                e = a.off[u + 1];
            }
        }
        int32_t found = -1;
        bu_stream_rows(a, Fp, i < qn && e > s, s, e, found, examined);
        if (i < qn && found >= 0) a.parent[u] = found;
    }
}

// MINB = blocks of BFS_THREADS per SM the register budget is sized for:
// 2 (64 registers, no spills) or 3 (40 registers, more warps to hide latency).
template <int MINB>
__global__ void __launch_bounds__(BFS_THREADS, MINB) bfs_kernel(BfsArgs a)
{
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    const unsigned lane = lane_id();
    const int64_t gwarp = gtid >> 5;
    const int64_t nwarps = gthreads >> 5;
    const int64_t n = a.n, nw = a.nw;
    WsHeader *h = a.hdr;
    const int32_t root = a.root;
    unsigned bar_target = grid_barrier_base(&h->bar);
    __shared__ WarpBuf s_wb[BFS_WARPS];
    __shared__ unsigned long long s_mf;
    WarpBuf &wb = s_wb[threadIdx.x >> 5];
    int qn_buf = 0, bn_buf = 0;  // warp-uniform fill levels of wb
    int un_open = 0;             // warp-uniform: vertices in this warp's open-list segment
    if (threadIdx.x == 0) s_mf = 0;
    unsigned long long my_mf = 0;

    // ---- init: bitmaps cleared, the root placed (the outputs are written
    // by the last pass; a vertex's state byte counts only once it is visited)
    for (int64_t w = gtid; w < nw; w += gthreads) {
        const unsigned rb = (w == (root >> 5)) ? 1u << (root & 31) : 0u;
        // isolated vertices (and ids >= n) start as visited: no search reaches
        // them and the bottom-up step need not test them; their outputs stay -1
        a.vis[w] = ~a.nz[w] | rb;
        a.fb[w] = rb;
        a.fb[nw + w] = 0;
        a.fb[2 * nw + w] = 0;
        a.fb[3 * nw + w] = 0;
    }
    if (gtid == 0) {
        const int64_t dr = a.off[root + 1] - a.off[root];
        a.parent[root] = root;
        mark_reached(a, root, 0, false);
        a.queue[0] = root;
        h->ctl[0].qcnt = 1;
        h->ctl[0].mf = (unsigned long long)dr;
        if (dr > a.big_deg) {
            h->ctl[0].big = (1ull << 32) | nchunks(dr);
            BigEnt be;
            be.u = root;
            be.cbase = 0;
            a.bigq[0] = be;
        }
    }
    if (!grid_sync(&h->bar, bar_target, a.st, a.timeout_ns, SITE_BFS_BAR)) return;
    if (gtid == 0) {
        h->t0 = globaltimer_ns();
        a.stats->init_ns = 0;
    }

    int64_t qbase = 0, bbase = 0, prev_qn = 0;
    double mu = (double)a.nnz;
    bool td = true, prev_td = true;
    unsigned long long my_edges = 0, my_touched = 0;
    int l = 0;
    for (;; ++l) {
        LevelCtl *cur = &h->ctl[l & 3];
        const int64_t qn = (int64_t)ldcg_u64(&cur->qcnt);
        if (qn == 0) break;
        if (l > n) {
            if (gtid == 0) record_error(a.st, GB_ERR_TIMEOUT, SITE_BFS_LEVELS, l);
            break;
        }
        const double mf = (double)ldcg_u64(&cur->mf);
        const unsigned long long bigp = ldcg_u64(&cur->big);
        const int64_t nb = (int64_t)(bigp >> 32);
        const int64_t nc = (int64_t)(bigp & 0xffffffffull);
        mu -= mf;
        if (l > 0) {
            if (td) {
                if (mf > mu / a.alpha) td = false;
            } else if (qn < prev_qn && (double)qn < (double)n / a.beta) {
                td = true;
            }
        }
        unsigned *F = a.fb + (size_t)(l & 3) * nw;
        unsigned *Fn = a.fb + (size_t)((l + 1) & 3) * nw;
        unsigned *Fz = a.fb + (size_t)((l + 2) & 3) * nw;
        unsigned *Fp = a.fb + (size_t)((l + 3) & 3) * nw;
        LevelCtl *nxt = &h->ctl[(l + 1) & 3];
        const int64_t qnext_base = qbase + qn;
        const int64_t bnext_base = bbase + nb;

        // Clear the bitmap and control record that level l+1 will fill.
        for (int64_t w = gtid; w < nw; w += gthreads) Fz[w] = 0;
        if (gtid == 0) {
            LevelCtl z = {0, 0, 0, 0};
            h->ctl[(l + 2) & 3] = z;
        }

        // Canonical parents of vertices claimed top-down at level l-1.
        if (a.canonical && l > 0 && prev_td) canonical_rescan(a, Fp, qbase, qn, gwarp, nwarps);

        if (td) {
            // (a) chunks of big frontier vertices, a contiguous range per warp
            if (nc > 0) {
                const int64_t per = (nc + nwarps - 1) / nwarps;
                const int64_t c0 = gwarp * per;
                const int64_t c1 = c0 + per < nc ? c0 + per : nc;
                if (c0 < c1) {
                    int64_t lo = 0, hi = nb;  // largest i with cbase(i) <= c0
                    while (hi - lo > 1) {
                        const int64_t mid = (lo + hi) >> 1;
                        if ((int64_t)load_big(a.bigq, bbase + mid).cbase <= c0) lo = mid;
                        else hi = mid;
                    }
                    int64_t ow = lo;
                    BigEnt be = load_big(a.bigq, bbase + ow);
                    for (int64_t c = c0; c < c1; ++c) {
                        while (ow + 1 < nb && (int64_t)load_big(a.bigq, bbase + ow + 1).cbase <= c) {
                            ++ow;
                            be = load_big(a.bigq, bbase + ow);
                        }
                        if (!GB_OK_IDX(a.st, be.u, a.n, 206)) continue;
                        const int64_t su = a.off[be.u], eu = a.off[be.u + 1];
                        const int64_t cs = (su & ~int64_t(3)) + (c - (int64_t)be.cbase) * BIG_CHUNK;
                        const int64_t s = su > cs ? su : cs;
                        const int64_t e = cs + BIG_CHUNK < eu ? cs + BIG_CHUNK : eu;
                        if (s >= e) continue;  // the empty chunk a row may end with
                        if (lane == 0) my_edges += (unsigned long long)(e - s);
                        // lane i: entries cs + 4i .. cs + 4i + 3, one 16-byte load when
                        // the column array allows it (the library's own graphs)
                        const int64_t j0 = cs + 4 * (int64_t)lane;
                        bool valid[TD_E];
                        int32_t sv[TD_E], vv[TD_E];
                        if (a.vec_col) {
                            int4 x = make_int4(0, 0, 0, 0);
                            if (j0 < e && GB_OK_IDX(a.st, j0 + 3, col_alloc_entries(a.nnz), 207))
                                x = __ldg(reinterpret_cast<const int4 *>(a.col + j0));
                            vv[0] = x.x;
                            vv[1] = x.y;
                            vv[2] = x.z;
                            vv[3] = x.w;
#pragma unroll
                            for (int t = 0; t < TD_E; ++t) valid[t] = j0 + t >= s && j0 + t < e;
                        } else {
#pragma unroll
                            for (int t = 0; t < TD_E; ++t) {
                                valid[t] = j0 + t >= s && j0 + t < e && GB_OK_IDX(a.st, j0 + t, a.nnz, 207);
                                vv[t] = valid[t] ? __ldg(&a.col[j0 + t]) : 0;
                            }
                        }
#pragma unroll
                        for (int t = 0; t < TD_E; ++t) sv[t] = be.u;
                        td_visit(valid, sv, vv, l, a, Fn, wb, qn_buf, bn_buf, my_mf, nxt,
                                 qnext_base, bnext_base);
                    }
                }
            }
            // (b) the other frontier vertices, 32 per warp, edges gathered as one stream
            for (int64_t i0 = gwarp * 32; i0 < qn; i0 += nwarps * 32) {
                const int64_t i = i0 + lane;
                int32_t u = 0;
                int64_t s = 0, d = 0;
                if (i < qn && GB_OK_IDX(a.st, qbase + i, a.n, 208)) {
                    u = ldcg_i32(&a.queue[qbase + i]);
                    if (!GB_OK_IDX(a.st, u, a.n, 209)) u = 0;
                    s = a.off[u];
                    d = a.off[u + 1] - s;
                    if (d > a.big_deg) d = 0;
                }
                const int64_t incl = warp_inclusive_scan(d);
                const int64_t total = __shfl_sync(kFull, incl, 31);
                const int64_t excl = incl - d;
                my_edges += d;
                my_touched += (i < qn);
                for (int64_t b = 0; b < total; b += 32 * TD_E) {
                    bool valid[TD_E];
                    int32_t sv[TD_E], vv[TD_E];
#pragma unroll
                    for (int t = 0; t < TD_E; ++t) {
                        const int64_t k = b + t * 32 + lane;
                        int owner = 0;
#pragma unroll
                        for (int step = 16; step >= 1; step >>= 1) {
                            const int cand = owner + step;
                            const int64_t ex = __shfl_sync(kFull, excl, cand);
                            if (ex <= k) owner = cand;
                        }
                        sv[t] = __shfl_sync(kFull, u, owner);
                        const int64_t so = __shfl_sync(kFull, s, owner);
                        const int64_t eo = __shfl_sync(kFull, excl, owner);
                        valid[t] = k < total && GB_OK_IDX(a.st, so + (k - eo), a.nnz, 210);
                        vv[t] = valid[t] ? __ldg(&a.col[so + (k - eo)]) : 0;
                    }
                    td_visit(valid, sv, vv, l, a, Fn, wb, qn_buf, bn_buf, my_mf, nxt, qnext_base,
                             bnext_base);
                }
            }
        } else {
            // bottom-up.  Hub pass: every open vertex tests its hub (fast mode),
            // a neighbour of largest degree, against the frontier bitmap; a hit
            // is its parent.  The vertices left open queue up in the warp's
            // pending ring, and every 32 of them take a row pass (one vertex per
            // lane), so the row probes run with full warps.  Vertices the row
            // pass leaves open go to the open list.  A bottom-up level that
            // follows another walks that list, 128 vertices per warp step, with
            // no bitmap scan and no visited test (only the lane holding a vertex
            // can visit it now); otherwise the warp walks its words of the
            // visited bitmap, BU_WORDS words (lane i: vertex i of each) per step,
            // and bulk-prefetches the next step's hub entries and row offsets
            // into L2 (16-byte aligned arrays only: the library's own are; a
            // caller's offsets may not be).
            int ph = 0, pt = 0;  // warp-uniform head and tail of the pending ring
            int32_t *seg = a.ulist ? a.ulist + gwarp * a.useg : nullptr;
            const bool from_seg = seg && l > 0 && !prev_td;   // the open list of the previous level
            const bool from_nzl = seg && !from_seg && a.nzl;  // the graph's non-isolated vertices
            // a list walk: this warp's segment (its own entries, in steps of
            // 32 * BU_WORDS), or the non-isolated list (steps strided over the
            // grid, a visited test per entry: top-down levels visited some)
            const int32_t *L = from_seg ? seg : a.nzl;
            const int64_t lcnt = from_seg ? un_open : a.nnzv;
            const int64_t lstart = from_seg ? 0 : gwarp * 32 * BU_WORDS;
            const int64_t lstride = from_seg ? 32 * BU_WORDS : nwarps * 32 * BU_WORDS;
            un_open = 0;
            const bool bulk_pf = !from_seg && !from_nzl && ((reinterpret_cast<uintptr_t>(a.off) |
                                                             reinterpret_cast<uintptr_t>(a.hub)) & 15u) == 0;
            if (from_seg || from_nzl) {
            for (int64_t i0 = lstart; i0 < lcnt; i0 += lstride) {
                int32_t u[BU_WORDS], dg[BU_WORDS], hb[BU_WORDS];
                bool cand[BU_WORDS];
#pragma unroll
                for (int t = 0; t < BU_WORDS; ++t) {
                    const int64_t i = i0 + t * 32 + lane;
                    cand[t] = i < lcnt;
                    u[t] = cand[t] ? ldcg_i32(&L[i]) : 0;
                    cand[t] = cand[t] && GB_OK_IDX(a.st, u[t], a.n, 232);
                }
                unsigned vw[BU_WORDS];
#pragma unroll
                for (int t = 0; t < BU_WORDS; ++t) {
                    vw[t] = cand[t] && from_nzl ? ldcg_u32(&a.vis[(unsigned)u[t] >> 5]) : 0u;
                    // hub and degree in one 8-byte load, not two scattered offsets
                    const int2 x = cand[t] ? __ldg(&a.hd[u[t]]) : make_int2(-1, 0);
                    dg[t] = x.y;
                    hb[t] = a.hub ? x.x : -1;
                }
#pragma unroll
                for (int t = 0; t < BU_WORDS; ++t) {
                    if (dg[t] == 65535)  // saturated: the exact degree from the offsets
                        dg[t] = (int32_t)(__ldg(&a.off[u[t] + 1]) - __ldg(&a.off[u[t]]));
                    if ((vw[t] >> (u[t] & 31)) & 1u) {  // visited by a top-down level
                        cand[t] = false;
                        hb[t] = -1;
                    }
                }
                unsigned fh[BU_WORDS];
#pragma unroll
                for (int t = 0; t < BU_WORDS; ++t)
                    fh[t] = hb[t] >= 0 && GB_OK_IDX(a.st, hb[t], a.n, 233) ? ldcg_u32(&F[hb[t] >> 5]) : 0u;
#pragma unroll
                for (int t = 0; t < BU_WORDS; ++t) {
                    const bool won = hb[t] >= 0 && ((fh[t] >> (hb[t] & 31)) & 1u);
                    my_touched += (unsigned)cand[t];
                    my_edges += (unsigned long long)(hb[t] >= 0);
                    if (won) mark_reached(a, u[t], l + 1, true);
                    set_bits(won, u[t], a.vis, Fn);
                    append_next(won, u[t], dg[t], a, wb, qn_buf, bn_buf, my_mf, nxt, qnext_base, bnext_base);
                    // a row of one entry was settled by the hub test: still open
                    const bool whole = hb[t] >= 0 && dg[t] == 1;
                    append_open(cand[t] && !won && whole, u[t], seg, un_open);
                    const bool pend = cand[t] && !won && !whole;
                    const unsigned pm = __ballot_sync(kFull, pend);
                    if (pend) wb.pu[(pt + __popc(pm & lanemask_lt())) & (PBUF - 1)] = u[t];
                    pt += __popc(pm);
                }
                while (pt - ph >= 32) {
                    bu_row_pass(a, F, Fn, ph, 32, l, wb, qn_buf, bn_buf, seg, un_open, my_mf, my_edges,
                                nxt, qnext_base, bnext_base);
                    ph += 32;
                }
            }
            } else {
            // this warp's words of the visited bitmap, BU_WORDS per step
            for (int64_t w0 = gwarp * BU_WORDS; w0 < nw; w0 += nwarps * BU_WORDS) {
                const int64_t wn = w0 + nwarps * BU_WORDS;
                if (bulk_pf && lane == 0 && (wn + BU_WORDS) * 32 <= n) {
                    if (a.hub) prefetch_l2_bulk(a.hub + wn * 32, BU_WORDS * 32 * sizeof(int32_t));
                    prefetch_l2_bulk(a.off + wn * 32, BU_WORDS * 32 * sizeof(int64_t));
                }
                unsigned vw[BU_WORDS];
                bool any = false;
#pragma unroll
                for (int t = 0; t < BU_WORDS; ++t) {
                    vw[t] = w0 + t < nw ? ldcg_u32(&a.vis[w0 + t]) : kFull;
                    any |= vw[t] != kFull;
                }
                if (!any) continue;
                int32_t dg[BU_WORDS], hb[BU_WORDS];
#pragma unroll
                for (int t = 0; t < BU_WORDS; ++t) {
                    const int64_t u = (w0 + t) * 32 + lane;
                    const bool cand = !((vw[t] >> lane) & 1u) && GB_OK_IDX(a.st, u, a.n, 216);
                    dg[t] = 0;
                    hb[t] = -1;
                    if (cand) {
                        dg[t] = (int32_t)(__ldg(&a.off[u + 1]) - __ldg(&a.off[u]));
                        if (a.hub) hb[t] = __ldg(&a.hub[u]);
                    }
                }
                unsigned fh[BU_WORDS];
#pragma unroll
                for (int t = 0; t < BU_WORDS; ++t)
                    fh[t] = hb[t] >= 0 && GB_OK_IDX(a.st, hb[t], a.n, 220) ? ldcg_u32(&F[hb[t] >> 5]) : 0u;
#pragma unroll
                for (int t = 0; t < BU_WORDS; ++t) {
                    if (vw[t] == kFull) continue;  // a fully visited word (warp-uniform)
                    const int64_t w = w0 + t;
                    const int64_t u = w * 32 + lane;
                    const bool cand = !((vw[t] >> lane) & 1u) && u < n;
                    const int32_t found = hb[t] >= 0 && ((fh[t] >> (hb[t] & 31)) & 1u) ? hb[t] : -1;
                    my_touched += (unsigned)cand;
                    my_edges += (unsigned long long)(hb[t] >= 0);
                    const bool won = found >= 0;
                    if (won) mark_reached(a, u, l + 1, true);
                    // the warp owns word w: commit it with two plain stores
                    const unsigned nm = __ballot_sync(kFull, won);
                    if (nm && lane == 0) {
                        __stcg(&a.vis[w], vw[t] | nm);
                        __stcg(&Fn[w], nm);
                    }
                    append_next(won, (int32_t)u, dg[t], a, wb, qn_buf, bn_buf, my_mf, nxt, qnext_base, bnext_base);
                    // no row pass for an empty row, nor for a row of one entry (its hub)
                    const bool pend = cand && found < 0 && dg[t] > (hb[t] >= 0 ? 1 : 0);
                    const unsigned pm = __ballot_sync(kFull, pend);
                    if (pend) wb.pu[(pt + __popc(pm & lanemask_lt())) & (PBUF - 1)] = (int32_t)u;
                    pt += __popc(pm);
                }
                while (pt - ph >= 32) {
                    bu_row_pass(a, F, Fn, ph, 32, l, wb, qn_buf, bn_buf, seg, un_open, my_mf, my_edges,
                                nxt, qnext_base, bnext_base);
                    ph += 32;
                }
            }
            }
            if (pt > ph)
                bu_row_pass(a, F, Fn, ph, pt - ph, l, wb, qn_buf, bn_buf, seg, un_open, my_mf, my_edges,
                            nxt, qnext_base, bnext_base);
        }
        // end of level: flush the staged vertices and add the block's degree sum
        flush_queue(wb, qn_buf, a, nxt, qnext_base);
        flush_big(wb, bn_buf, a, nxt, bnext_base);
        {
            const unsigned long long t = warp_sum(my_mf);
            my_mf = 0;
            if (lane == 0 && t) atomicAdd(&s_mf, t);
            __syncthreads();
            if (threadIdx.x == 0) {
                if (s_mf) atomicAdd(&nxt->mf, s_mf);
                s_mf = 0;
            }
        }
        prev_td = td;
        prev_qn = qn;
        qbase += qn;
        bbase += nb;
        if (gtid == 0) atomicAdd(&h->acc[td ? 4 : 5], 1ull);
        if (!grid_sync(&h->bar, bar_target, a.st, a.timeout_ns, SITE_BFS_BAR)) return;
        if (gtid == 0 && l < kStatLevels) {
            const uint64_t now = globaltimer_ns();
            a.stats->level_ns[l] = now - h->t0;
            a.stats->level_frontier[l] = qn;
            a.stats->level_dir[l] = td ? 1 : 2;
            h->t0 = now;
        }
    }

    // ---- outputs: level and parent of every vertex, whole lines per warp.
    // Reached = visited and not isolated (isolated vertices start visited),
    // or the root; everyone else gets -1.  The state bytes, parents and
    // escaped levels were written by other blocks before the last barrier.
    // Each lane takes 4 consecutive vertices: one 4-byte load of their state
    // bytes, and the hub and parent entries loaded as 16-byte vectors at the
    // same time (not after the state bytes: one memory round trip per
    // group), so that a warp moves 128 vertices per step.
    if (a.vec_out) {
        for (int64_t g0 = gwarp * 128; g0 < n; g0 += nwarps * 128) {
            const int64_t v0 = g0 + 4 * (int64_t)lane;
            if (v0 + 3 < n) {
                const int64_t w = v0 >> 5;
                const unsigned sh = (unsigned)(v0 & 31);
                const unsigned rbits = ((ldcg_u32(&a.vis[w]) & __ldg(&a.nz[w])) >> sh) & 15u;
                const unsigned sw = __ldcg(reinterpret_cast<const unsigned *>(a.st8 + v0));
                const int4 hv = a.hub ? __ldg(reinterpret_cast<const int4 *>(a.hub + v0)) : make_int4(-1, -1, -1, -1);
                const int4 pv = __ldcg(reinterpret_cast<const int4 *>(a.parent + v0));
                int lv[4], pr[4];
                const int hh[4] = {hv.x, hv.y, hv.z, hv.w};
                const int pp[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const unsigned b = (sw >> (8 * t)) & 255u;
                    const bool reached = ((rbits >> t) & 1u) || v0 + t == root;
                    lv[t] = -1;
                    pr[t] = -1;
                    if (reached) {
                        lv[t] = (b & ST_ESC) == ST_ESC ? ldcg_i32(&a.level[v0 + t]) : (int32_t)(b & ST_ESC) - 1;
                        pr[t] = (b & ST_HUB) ? hh[t] : pp[t];
                    }
                }
                *reinterpret_cast<int4 *>(a.level + v0) = make_int4(lv[0], lv[1], lv[2], lv[3]);
                *reinterpret_cast<int4 *>(a.parent + v0) = make_int4(pr[0], pr[1], pr[2], pr[3]);
            } else {
                for (int64_t v = v0; v < n && v < v0 + 4; ++v) {
                    const bool reached = ((ldcg_u32(&a.vis[v >> 5]) & __ldg(&a.nz[v >> 5])) >> (v & 31) & 1u) ||
                                         v == root;
                    int32_t lvv = -1, prv = -1;
                    if (reached) {
                        const unsigned b = __ldcg(&a.st8[v]);
                        lvv = (b & ST_ESC) == ST_ESC ? ldcg_i32(&a.level[v]) : (int32_t)(b & ST_ESC) - 1;
                        prv = (b & ST_HUB) ? __ldg(&a.hub[v]) : ldcg_i32(&a.parent[v]);
                    }
                    a.level[v] = lvv;
                    a.parent[v] = prv;
                }
            }
        }
    } else {
        for (int64_t v = gtid; v < n; v += gthreads) {
            const bool reached = ((ldcg_u32(&a.vis[v >> 5]) & __ldg(&a.nz[v >> 5])) >> (v & 31) & 1u) ||
                                 v == root;
            int32_t lvv = -1, prv = -1;
            if (reached) {
                const unsigned b = __ldcg(&a.st8[v]);
                lvv = (b & ST_ESC) == ST_ESC ? ldcg_i32(&a.level[v]) : (int32_t)(b & ST_ESC) - 1;
                prv = (b & ST_HUB) ? __ldg(&a.hub[v]) : ldcg_i32(&a.parent[v]);
            }
            a.level[v] = lvv;
            a.parent[v] = prv;
        }
    }

    // ---- statistics: block partial sums, the last block publishes them
    my_edges = warp_sum(my_edges);
    my_touched = warp_sum(my_touched);
    if (lane == 0) {
        if (my_edges) atomicAdd(&h->acc[0], my_edges);
        if (my_touched) atomicAdd(&h->acc[1], my_touched);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&h->done, 1u);
        if (prev == gridDim.x - 1) {
            __threadfence();
            BfsDevStats &s = *a.stats;
            s.nlevels = (unsigned long long)l;
            s.edges_examined = ldcg_u64(&h->acc[0]);
            s.vertices_touched = ldcg_u64(&h->acc[1]);
            s.reached = (unsigned long long)qbase;
            s.td_levels = ldcg_u64(&h->acc[4]);
            s.bu_levels = ldcg_u64(&h->acc[5]);
        }
    }
}

}  // namespace

// The output pass uses 16-byte vector access when every array it touches
// allows it (a caller's outputs may start anywhere).
static int vec_ok(const BfsArgs &a)
{
    const uintptr_t m = reinterpret_cast<uintptr_t>(a.parent) | reinterpret_cast<uintptr_t>(a.level) |
                        reinterpret_cast<uintptr_t>(a.hub) | reinterpret_cast<uintptr_t>(a.st8);
    return (m & 15u) == 0 ? 1 : 0;
}

int bfs_pick_blocks(int num_sms, int minb)
{
    int per_sm = 0;
    const void *k = minb == 2 ? (const void *)bfs_kernel<2> : (const void *)bfs_kernel<3>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, BFS_THREADS, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    return num_sms * std::min(per_sm, minb);
}

namespace {
// Entries of the open list: every warp of the grid gets a segment for the
// vertices of its bitmap words (it owns BU_WORDS words of every
// nwarps * BU_WORDS), i.e. n rounded up per warp; room for grids of up to
// kOpenMaxWarps warps.
constexpr int64_t kOpenMaxWarps = 8192;
int64_t open_list_cap(int64_t n) { return ((n + 31) / 32) * 32 + kOpenMaxWarps * 32 * BU_WORDS; }

// Segment length per warp for a grid of nwarps warps, or 0 if the list cannot
// hold them (the search then walks the bitmap at every bottom-up level).
int64_t open_list_seg(int64_t n, int64_t nwarps)
{
    const int64_t nw = (n + 31) / 32;
    const int64_t steps = (nw + nwarps * BU_WORDS - 1) / (nwarps * BU_WORDS);
    const int64_t seg = steps * BU_WORDS * 32;
    return seg * nwarps <= open_list_cap(n) ? seg : 0;
}

struct WsLayout {
    size_t off_vis, off_fb, off_q, off_st, off_ul, off_big, total;
    int64_t bigcap;
};
// one buffer: header | visited | 4 frontier bitmaps | queue | state bytes |
// open list | big list
WsLayout ws_layout(const gb_graph *g, int big_deg)
{
    WsLayout L;
    const int64_t n = g->n, nw = (n + 31) / 32;
    L.bigcap = g->nnz / (big_deg + 1) + 2;
    L.off_vis = (sizeof(WsHeader) + 255) & ~size_t(255);
    L.off_fb = L.off_vis + ((nw * 4 + 255) & ~size_t(255));
    L.off_q = L.off_fb + ((4 * nw * 4 + 255) & ~size_t(255));
    L.off_st = L.off_q + ((n * 4 + 255) & ~size_t(255));
    L.off_ul = L.off_st + ((nw * 32 + 255) & ~size_t(255));
    L.off_big = L.off_ul + ((open_list_cap(n) * 4 + 255) & ~size_t(255));
    L.total = L.off_big + L.bigcap * sizeof(BigEnt);
    return L;
}
}  // namespace

size_t bfs_workspace_bytes(const gb_graph *g)
{
    return ws_layout(g, 1).total;  // big_degree 1 is the largest big list
}

gb_status bfs_impl(const gb_graph *g, int64_t root, int32_t *parent, int32_t *level,
                   BfsDevStats *stats, cudaStream_t s, int grid, unsigned char *given_ws)
{
    Context *ctx = context();
    if (!ctx) return GB_ERR_CUDA;
    const gb_bfs_options &o = options();
    const int64_t n = g->n;
    const int64_t nw = (n + 31) / 32;
    const int big_deg = std::max(o.big_degree, 1);
    const WsLayout Lw = ws_layout(g, big_deg);
    const int64_t bigcap = Lw.bigcap;
    const size_t off_vis = Lw.off_vis, off_fb = Lw.off_fb, off_q = Lw.off_q, off_big = Lw.off_big;
    unsigned char *ws = given_ws;
    Scratch tmp(s);
    if (!ws) GB_CUDA(tmp.alloc(&ws, Lw.total));
    GB_CUDA(cudaMemsetAsync(ws, 0, sizeof(WsHeader), s));
    BfsArgs a;
    a.off = g->off;
    a.col = g->col;
    a.nz = g->nz;
    // the hub test finds some parent, not the smallest-id one
    a.hub = o.canonical_parents ? nullptr : g->hub;
    a.n = n;
    a.nnz = g->nnz;
    a.root = (int32_t)root;
    a.parent = parent;
    a.level = level;
    a.hdr = reinterpret_cast<WsHeader *>(ws);
    a.vis = reinterpret_cast<unsigned *>(ws + off_vis);
    a.fb = reinterpret_cast<unsigned *>(ws + off_fb);
    a.nw = nw;
    a.queue = reinterpret_cast<int32_t *>(ws + off_q);
    a.st8 = ws + Lw.off_st;
    a.ulist = reinterpret_cast<int32_t *>(ws + Lw.off_ul);
    a.nzl = g->nzl;
    a.nnzv = g->nnzv;
    a.hd = g->hd;
    a.bigq = reinterpret_cast<BigEnt *>(ws + off_big);
    a.bigcap = bigcap;
    a.st = ctx->status;
    a.stats = stats;
    a.alpha = (float)o.alpha;
    a.beta = (float)o.beta;
    a.big_deg = big_deg;
    a.canonical = o.canonical_parents;
    a.vec_out = vec_ok(a);
    a.vec_col = (reinterpret_cast<uintptr_t>(a.col) & 15u) == 0;  // allocated with col_alloc_entries
    a.timeout_ns = timeout_ns();
    void *args[] = {&a};
    // 1 block per SM runs the 2-per-SM kernel on half its grid
    const int minb = o.blocks_per_sm == 3 ? 3 : 2;
    const int full = minb == 3 ? ctx->bfs_blocks
                               : (o.blocks_per_sm == 1 ? std::max(1, ctx->bfs_blocks2 / 2) : ctx->bfs_blocks2);
    const int blocks = grid > 0 && grid < full ? grid : full;
    a.useg = open_list_seg(n, (int64_t)blocks * (BFS_THREADS / 32));
    if (a.useg == 0 || !a.hd) a.ulist = nullptr;  // the list walks read hd
    const void *kern = minb == 2 ? (const void *)bfs_kernel<2> : (const void *)bfs_kernel<3>;
    GB_CUDA(cudaLaunchCooperativeKernel(kern, dim3(blocks),
                                        dim3(BFS_THREADS), args, 0, s));
    note_launch();
    return GB_OK;
}

}  // namespace gb

// ---------------------------------------------------------------------------
// bfs_noalloc: the single-source BFS kernel above, for callers that cannot
// allocate device memory.  Its scratch lives in one file-scope device array
// sized for graphs of up to 2^20 vertices; nothing here calls cudaMalloc,
// cudaMallocAsync or cudaFree.
// ---------------------------------------------------------------------------
namespace gb {
namespace {

constexpr int64_t kNaMaxN = int64_t(1) << 20;      // largest graph (vertices)
constexpr int64_t kNaWords = kNaMaxN / 32;
constexpr int64_t kNaBigCap = kNaMaxN + 2;         // a vertex enters the big list at most once
constexpr size_t kNaHdr = 0;
constexpr size_t kNaVis = 1024;
constexpr size_t kNaFb = kNaVis + kNaWords * 4;
constexpr size_t kNaNz = kNaFb + 4 * kNaWords * 4;
constexpr size_t kNaQueue = kNaNz + kNaWords * 4;
constexpr size_t kNaSt = kNaQueue + kNaMaxN * 4;
constexpr size_t kNaBig = kNaSt + kNaMaxN;
constexpr size_t kNaStatus = kNaBig + kNaBigCap * sizeof(BigEnt);
constexpr size_t kNaStats = kNaStatus + 256;
constexpr size_t kNaBytes = kNaStats + ((sizeof(BfsDevStats) + 255) & ~size_t(255));
static_assert(sizeof(WsHeader) <= kNaVis - kNaHdr, "header region too small");
static_assert(sizeof(DevStatus) <= 256, "status region too small");

// Shared by every call on a device; the last call's contents stay behind.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Bit v of word v/32: row v is not empty (computed into the scratch).
__global__ void na_nz_kernel(const int64_t *__restrict__ off, int64_t n, uint32_t *__restrict__ nz,
                             int64_t nw)
{
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned lane = threadIdx.x & 31u;
    for (int64_t w = gw; w < nw; w += stride) {
        const int64_t v = w * 32 + lane;
        const bool has = v < n && off[v + 1] > off[v];
        const unsigned b = __ballot_sync(kFull, has);
        if (lane == 0) nz[w] = b;
    }
}

struct NoAllocDevice {
    bool ready = false;
    unsigned char *scratch = nullptr;  // device address of g_noalloc_scratch
    int num_sms = 0;
    int blocks = 0;
};
std::mutex g_na_mu;
NoAllocDevice g_na[64];

}  // namespace

gb_status bfs_noalloc_impl(const int64_t *off, const int32_t *col, int64_t n, int64_t nnz,
                           int64_t root, int32_t *parent, int32_t *level, cudaStream_t s)
{
    if (!off || !parent || !level || (nnz > 0 && !col) || n < 1 || nnz < 0) {
        set_error("bfs_noalloc: need off, parent, level (and col when nnz > 0), n >= 1");
        return GB_ERR_INVALID;
    }
    if (n > kNaMaxN) {
        set_error("bfs_noalloc: the graph has more than 2^20 vertices, the size of the "
                  "built-in scratch; use bfs() instead");
        return GB_ERR_RANGE;
    }
    if (root < 0 || root >= n) {
        set_error("bfs_noalloc: root outside [0, n)");
        return GB_ERR_RANGE;
    }
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("bfs_noalloc: device index above 63");
        return GB_ERR_INVALID;
    }
    NoAllocDevice d;
    {
        // One-time set-up per device, with that device current: the device
        // address of the scratch array and the cooperative grid size.
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na[dev].ready) {
            NoAllocDevice nd;
            GB_CUDA(cudaGetSymbolAddress((void **)&nd.scratch, g_noalloc_scratch));
            GB_CUDA(cudaDeviceGetAttribute(&nd.num_sms, cudaDevAttrMultiProcessorCount, dev));
            int per_sm = 0;
            GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bfs_kernel<2>,
                                                                  BFS_THREADS, 0));
            nd.blocks = nd.num_sms * std::max(1, std::min(per_sm, 2));
            nd.ready = true;
            g_na[dev] = nd;
        }
        d = g_na[dev];
    }
    const gb_bfs_options &o = options();
    const int64_t nw = (n + 31) / 32;
    unsigned char *ws = d.scratch;
    // The header (barrier, level counters) and the status word must start at zero.
    GB_CUDA(cudaMemsetAsync(ws + kNaHdr, 0, sizeof(WsHeader), s));
    GB_CUDA(cudaMemsetAsync(ws + kNaStatus, 0, sizeof(DevStatus), s));
    na_nz_kernel<<<d.num_sms * 4, 256, 0, s>>>(off, n, reinterpret_cast<uint32_t *>(ws + kNaNz), nw);
    note_launch();
    GB_CUDA(cudaGetLastError());
    BfsArgs a;
    a.off = off;
    a.col = col;
    a.nz = reinterpret_cast<const uint32_t *>(ws + kNaNz);
    a.hub = nullptr;
    a.n = n;
    a.nnz = nnz;
    a.root = (int32_t)root;
    a.parent = parent;
    a.level = level;
    a.hdr = reinterpret_cast<WsHeader *>(ws + kNaHdr);
    a.vis = reinterpret_cast<unsigned *>(ws + kNaVis);
    a.fb = reinterpret_cast<unsigned *>(ws + kNaFb);
    a.nw = nw;
    a.queue = reinterpret_cast<int32_t *>(ws + kNaQueue);
    a.st8 = ws + kNaSt;
    a.ulist = nullptr;  // no open list: every bottom-up level walks the bitmap
    a.useg = 0;
    a.nzl = nullptr;
    a.nnzv = 0;
    a.hd = nullptr;
    a.bigq = reinterpret_cast<BigEnt *>(ws + kNaBig);
    a.bigcap = kNaBigCap;
    a.st = reinterpret_cast<DevStatus *>(ws + kNaStatus);
    a.stats = reinterpret_cast<BfsDevStats *>(ws + kNaStats);
    a.alpha = (float)o.alpha;
    a.beta = (float)o.beta;
    a.big_deg = std::max(o.big_degree, 1);
    a.canonical = o.canonical_parents;
    a.vec_out = vec_ok(a);
    a.vec_col = 0;  // a caller's columns: neither alignment nor padding is known
    a.timeout_ns = timeout_ns();
    void *args[] = {&a};
    GB_CUDA(cudaLaunchCooperativeKernel((const void *)bfs_kernel<2>, dim3(d.blocks),
                                        dim3(BFS_THREADS), args, 0, s));
    note_launch();
    DevStatus hst;
    GB_CUDA(cudaMemcpyAsync(&hst, ws + kNaStatus, sizeof(hst), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    if (hst.code != 0) {
        set_error("bfs_noalloc: device status " + std::to_string(hst.code) + " at site " +
                  std::to_string(hst.where));
        return (gb_status)hst.code;
    }
    return GB_OK;
}

}  // namespace gb

extern "C" gb_status bfs_noalloc(const int64_t *off, const int32_t *col, int64_t n, int64_t nnz,
                                 int64_t root, int32_t *parent, int32_t *level, gb_stream s)
{
    try {
        return gb::bfs_noalloc_impl(off, col, n, nnz, root, parent, level,
                                    reinterpret_cast<cudaStream_t>(s));
    } catch (...) {
        gb::set_error("bfs_noalloc: internal error");
        return GB_ERR_INVALID;
    }
}
