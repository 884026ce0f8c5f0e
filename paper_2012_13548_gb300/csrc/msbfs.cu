// Batched kernel 2: multi-source BFS with per-vertex bitmask frontiers.
//
// Bit b of a vertex mask belongs to root b.  A level of every search is one
// level of Algorithm "Parallel BFS" (Sec. 2.3.2) applied to all bits at once
// (the multi-source traversal of Then et al., VLDB 2014): the frontier of
// vertex v is M_l[v] (bits whose level at v is l), seen[v] holds the bits
// with level <= l.  Bits are independent, so every row of the result equals
// the single-source result of its root.
//
//  top-down level: (1) every active vertex v ORs M_l[v] & ~seen[u] into
//    M_{l+1}[u] for its neighbours u (one atomic per edge that adds bits);
//    the first writer of a vertex appends it to the next active list, and
//    the bits an atomic sets first have v as a valid parent, which is
//    written there unless canonical parents are asked for; (2) after a grid
//    barrier, in canonical mode, each new vertex scans its sorted adjacency
//    list for, per new bit, the first neighbour carrying that bit in M_l --
//    the smallest-id parent -- and writes levels and parents.
//  bottom-up level: every vertex with unseen bits scans its sorted adjacency
//    list, collecting M_l bits until all its unseen bits are found; the first
//    neighbour to supply a bit is its parent.  A warp takes 32 consecutive
//    vertices and streams their rows together, every open row getting an
//    equal share of 32 lanes x 4 consecutive entries per round; a segmented
//    prefix-OR over the lanes credits each bit to its first (smallest-id)
//    neighbour.  On the first bottom-up level after top-down ones nearly every
//    row is scanned to its end, so rows longer than MS_HUGE entries (listed
//    once per batch call) are scanned first, one per warp, and the groups of
//    32 are then handed out by a counter: a warp that drew a long row takes
//    fewer groups, instead of holding the level barrier.
//
// Outputs of batch calls: as bits are found their parents and levels go to
// vertex-major staging arrays ([n][k]: the bits of one vertex share a few
// cache lines), and after the last level the same kernel writes the [k][n]
// outputs from them, every entry once (-1 where the vertex's seen mask lacks
// the bit).  Written straight into the [k][n] rows, each found bit was its
// own partially written sector in a different row; that cost ~70% of a
// 64-root search.
//
// The same kernel runs a batch of graphs: vertex ids are made global by
// per-graph offsets, every graph's roots use the low bits, and since the
// graphs share no edges their searches cannot mix.  Masks are uint64 for up
// to 64 roots of one graph and uint8 for up to 8 roots per graph of a batch.
//
// Serving runs the same kernel one level per launch on a resident graph: the
// search state stays in a per-graph workspace between launches, queries take
// free bits at level boundaries (a per-slot table gives each bit its own
// output buffers and the level it started at), and the kernel reports which
// bits still advance so the host can retire finished queries.
#include "common.cuh"
#include "internal.h"

#include <algorithm>
#include <mutex>
#include <vector>

namespace gb {
namespace {

constexpr int MS_THREADS = 512;
constexpr int MS_MAXG = 64;
constexpr int MS_BIG_CHUNK = 256;
constexpr int MS_BIG_DEG = 256;
constexpr int MS_WARPS = MS_THREADS / 32;
constexpr int MS_QBUF = 256;  // per-warp staging of newly active vertices
constexpr int MS_BBUF = 32;   // per-warp staging of newly active big vertices
constexpr int MS_HIST = 8;    // batch calls: levels whose reached-bit masks are kept
constexpr int MS_HUGE = 4096; // bottom-up: rows longer than this are scanned first, one per warp
// batch calls on graphs of at least this many vertices (frontier masks of
// 256 MB and more, twice the L2) run on the graph's degree-ordered copy; at
// 2^24 vertices the copy measured slower, at 2^26 faster
constexpr int64_t MS_LAYOUT_MIN_N = int64_t(1) << 25;
constexpr int SITE_MS_BAR = 30;
constexpr int SITE_MS_LEVELS = 31;

struct MsGraph {
    const int64_t *off;
    const int32_t *col;
    const uint32_t *nz;  // degree >= 1 bitmap
    int64_t voff;  // first global id
    int64_t n;
    int32_t *par;  // [k][n]
    int32_t *lev;  // [k][n]
    int32_t *pst;  // batch calls: parents staged vertex-major, [n][kst]
    int32_t *lst;  // and levels
    int64_t kst;
    // the search runs on the graph's degree-ordered copy (off/col above are the
    // copy's): ids inside the kernel are copy ids, perm maps them back and inv
    // maps the roots in; both null when the search runs on the graph itself
    const int32_t *perm;
    const int32_t *inv;
};

}  // namespace

struct MsHeader {
    GridBarrier bar;
    unsigned done;
    unsigned pad0;
    MsCtl ctl[3];
    unsigned long long acc[6];
    unsigned long long na_hist[4];  // active-list length of each level (ring)
    unsigned long long t0;          // global timer at the start of the current level
    unsigned long long gnext[4];    // bottom-up: next group of 32 vertices (ring by level)
    unsigned long long nhuge;       // entries of the huge-row list
};

namespace {

template <typename T>
struct MsArgs {
    const MsGraph *graphs;  // device [ng]
    int ng;
    int k;                  // bits in use
    int64_t ntot;           // sum of n over graphs
    int64_t mstride;        // ntot rounded up to 64: distance between mask buffers
    int64_t nnz_tot;
    const int64_t *roots;   // device [ng][k]: local root ids
    T *seen;
    T *mbuf;                // 3 masks of ntot (ring)
    T *hist;                // batch calls: bits first reached at levels 0..MS_HIST-1,
                            // [MS_HIST][mstride]; nullptr in serving
    int32_t *act;           // 3 active lists of ntot (ring)
    unsigned long long *bigq;  // chunk list of big active vertices (gid | cbase << 32)
    int64_t bigcap;
    MsHeader *hdr;
    DevStatus *st;
    BfsDevStats *stats;     // nullptr: no statistics (serving)
    float ms_alpha;
    float ms_beta;
    uint64_t timeout_ns;
    int canonical;          // 1: smallest-id parents; 0: any valid parent
    int l0;                 // first level to run
    int max_levels;         // levels to run in this launch, 0 = until the frontier is empty
    int do_init;            // 1: clear state and place the roots first (batch calls)
    unsigned long long active;  // serving: bits in use; ignored when do_init
    const MsSlots *slots;   // serving: per-bit outputs; nullptr = graph outputs [k][n]
    int vec_col;            // 1: every graph's column array is 16-byte aligned and padded
    int32_t *huge;          // single-graph batch calls: vertices of degree > MS_HUGE (else null)
};

template <typename T>
__device__ __forceinline__ T ld_mask(const T *p);
template <>
__device__ __forceinline__ unsigned long long ld_mask(const unsigned long long *p)
{
    return __ldcg(p);
}
template <>
__device__ __forceinline__ unsigned char ld_mask(const unsigned char *p)
{
    return __ldcg(p);
}

template <typename T>
__device__ __forceinline__ T atomic_or_mask(T *p, T m);
template <>
__device__ __forceinline__ unsigned long long atomic_or_mask(unsigned long long *p,
                                                              unsigned long long m)
{
    return atomicOr(p, m);
}
template <>
__device__ __forceinline__ unsigned char atomic_or_mask(unsigned char *p, unsigned char m)
{
    unsigned *w = reinterpret_cast<unsigned *>(reinterpret_cast<uintptr_t>(p) & ~uintptr_t(3));
    const unsigned sh = (unsigned)(reinterpret_cast<uintptr_t>(p) & 3u) * 8u;
    const unsigned old = atomicOr(w, (unsigned)m << sh);
    return (unsigned char)(old >> sh);
}

template <typename T>
__device__ __forceinline__ void st_mask(T *p, T v)
{
    *reinterpret_cast<volatile T *>(p) = v;
}

template <typename T>
__device__ __forceinline__ T shfl_mask(T v, int src)
{
    return (T)__shfl_sync(kFull, (unsigned long long)v, src);
}
template <typename T>
__device__ __forceinline__ T shfl_up_mask(T v, int d)
{
    return (T)__shfl_up_sync(kFull, (unsigned long long)v, d);
}

// OR of the masks of lanes below this one.
template <typename T>
__device__ __forceinline__ T warp_exclusive_or(T v)
{
    const unsigned lane = lane_id();
    T incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T t = shfl_up_mask(incl, o);
        if (lane >= (unsigned)o) incl |= t;
    }
    const T ex = shfl_up_mask(incl, 1);
    return lane == 0 ? (T)0 : ex;
}

template <typename T>
__device__ __forceinline__ T warp_or(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v |= (T)__shfl_xor_sync(kFull, (unsigned long long)v, o);
    return v;
}

// graph index of global vertex id (graphs sorted by voff; s_voff has ng+1 entries)
__device__ __forceinline__ int find_graph(const int64_t *s_voff, int ng, int64_t gid)
{
    int lo = 0, hi = ng;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_voff[mid] <= gid) lo = mid;
        else hi = mid;
    }
    return lo;
}

// The original id of a vertex of the search (the identity unless the search
// runs on the degree-ordered copy).  The staged outputs (parents, levels, the
// level masks) are kept by original id, so the final pass reads them in line
// with its output rows.
__device__ __forceinline__ int64_t orig_id(const MsGraph &G, int64_t local)
{
    return G.perm ? (int64_t)__ldg(&G.perm[local]) : local;
}

// local: the vertex whose parents these are (already an original id if
// local_orig); p: the parent, an id of the search.
template <typename T>
__device__ __forceinline__ void write_parents(const MsGraph &G, const MsSlots *S, int64_t local,
                                              T bits, int32_t p, bool local_orig = false)
{
    if (!S && G.perm) {  // staged by original id, as an original id
        if (!local_orig) local = orig_id(G, local);
        p = (int32_t)orig_id(G, p);
    }
    if (!S && (G.kst & 15) == 0) {
        // an aligned group of 4 bits that all take this parent: one 16-byte store
        int32_t *row = G.pst + local * G.kst;
        unsigned long long bb = (unsigned long long)bits;
        while (bb) {
            const int b = __ffsll(bb) - 1;
            if ((b & 3) == 0 && ((bb >> b) & 15ull) == 15ull) {
                *reinterpret_cast<int4 *>(row + b) = make_int4(p, p, p, p);
                bb &= ~(15ull << b);
            } else {
                row[b] = p;
                bb &= bb - 1;
            }
        }
        return;
    }
    while (bits) {
        const int b = __ffsll((unsigned long long)bits) - 1;
        bits &= bits - 1;
        if (S) S->par[b][local] = p;
        else G.pst[local * G.kst + b] = p;
    }
}

// lvl = the global level number; a serving slot stores it relative to its start
template <typename T>
__device__ __forceinline__ void write_levels(const MsGraph &G, const MsSlots *S, int64_t local,
                                             T bits, int32_t lvl)
{
    if (!S && lvl < MS_HIST) return;  // earlier levels: the mask history
    if (!S && G.perm) local = orig_id(G, local);
    while (bits) {
        const int b = __ffsll((unsigned long long)bits) - 1;
        bits &= bits - 1;
        if (S) S->lev[b][local] = lvl - S->start[b];
        else G.lst[local * G.kst + b] = lvl;
    }
}

// Newly active vertices are staged per warp in shared memory and moved to the
// next active list with one atomic per flush; the fill levels qn/bn are
// warp-uniform registers (every lane adds the same ballot counts).
struct MsWarpBuf {
    int32_t q[MS_QBUF];
    unsigned long long b[MS_BBUF];  // gid | nchunks << 32
};

// Warp-collective: move the staged vertices to the next active list.
__device__ __forceinline__ void ms_flush_q(MsWarpBuf &wb, int &qn, MsCtl *nxt, int32_t *act_next)
{
    if (qn == 0) return;
    __syncwarp();
    const unsigned lane = lane_id();
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&nxt->na, (unsigned long long)qn);
    base = __shfl_sync(kFull, base, 0);
    for (int i = lane; i < qn; i += 32) __stcg(&act_next[base + i], wb.q[i]);
    __syncwarp();
    qn = 0;
}

// Warp-collective: chunk ranges for the staged big vertices.
__device__ __forceinline__ void ms_flush_b(MsWarpBuf &wb, int &bn, MsCtl *nxt,
                                           unsigned long long *bigq_next)
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
    if ((int)lane < bn) {
        const unsigned long long cb = (p & 0xffffffffull) + incl - nch;
        __stcg(&bigq_next[(int64_t)(p >> 32) + lane], (e & 0xffffffffull) | (cb << 32));
    }
    __syncwarp();
    bn = 0;
}

// Warp-collective: the lanes with `on` join the next active list.
__device__ __forceinline__ void ms_append(bool on, int64_t gid, int64_t deg, MsWarpBuf &wb,
                                          int &qn, int &bn, unsigned long long &my_mf, MsCtl *nxt,
                                          int32_t *act_next, unsigned long long *bigq_next)
{
    const unsigned bal = __ballot_sync(kFull, on);
    if (!bal) return;
    const int cnt = __popc(bal);
    if (qn + cnt > MS_QBUF) ms_flush_q(wb, qn, nxt, act_next);
    if (on) {
        wb.q[qn + __popc(bal & lanemask_lt())] = (int32_t)gid;
        my_mf += (unsigned long long)deg;
    }
    qn += cnt;
    const bool big = on && deg > MS_BIG_DEG;
    const unsigned bb = __ballot_sync(kFull, big);
    if (bb) {
        const int bc = __popc(bb);
        if (bn + bc > MS_BBUF) ms_flush_b(wb, bn, nxt, bigq_next);
        if (big)
            wb.b[bn + __popc(bb & lanemask_lt())] =
                (unsigned long long)(uint32_t)gid |
                ((unsigned long long)((deg + MS_BIG_CHUNK - 1) / MS_BIG_CHUNK) << 32);
        bn += bc;
    }
}

// Top-down expansion of one edge (gv -> gu) carrying frontier bits f.
// Top-down visit of edge (v, gu), v the frontier vertex (local id pv) with
// mask f.  The bits this atomic sets first are gu's new bits with v as their
// parent: outside canonical mode that parent and the level are written here,
// once per bit, and gu's row is never scanned for them.
template <typename T>
__device__ __forceinline__ void ms_td_edge(bool valid, T f, int64_t gu, int32_t pv, int l,
                                           const MsArgs<T> &a, const MsSlots *S, T *Mn,
                                           const MsGraph *s_g, const int64_t *s_voff, MsWarpBuf &wb,
                                           int &qn, int &bn, unsigned long long &my_mf,
                                           MsCtl *nxt, int32_t *act_next,
                                           unsigned long long *bigq_next)
{
    bool first = false;
    int64_t deg = 0;
    if (valid) {
        const T m = f & (T)~ld_mask(&a.seen[gu]);
        if (m) {
            const T old = atomic_or_mask(&Mn[gu], m);
            const T newb = m & (T)~old;
            if (old == 0 || (!a.canonical && newb)) {
                const int g = find_graph(s_voff, a.ng, gu);
                const int64_t lu = gu - s_g[g].voff;
                if (!a.canonical && newb) {
                    write_parents(s_g[g], S, lu, newb, pv);
                    write_levels(s_g[g], S, lu, newb, l + 1);
                }
                if (old == 0) {
                    first = true;
                    deg = s_g[g].off[lu + 1] - s_g[g].off[lu];
                }
            }
        }
    }
    ms_append(first, gu, deg, wb, qn, bn, my_mf, nxt, act_next, bigq_next);
}

// Rows of a warp (lane i owns one row: graph g, adjacency [s, e), missing
// bits `need`; lu is the row's vertex as the staged outputs know it, its
// original id) are scanned together.  Each round deals 4 x 32
// neighbour slots, an equal share to every row still missing bits, so a row
// that completes early stops taking slots; the loads of a round are issued
// together.  Slots are processed in neighbour order: a segmented prefix-OR
// over the slots of each row credits every bit to the first neighbour that
// carries it in M, which is the smallest-id parent.  Returns the bits found
// for this lane's row (parents written).
template <typename T>
__device__ __forceinline__ T ms_rows(const MsGraph *s_g, const MsSlots *S, const T *M, int g,
                                     int64_t lu, int64_t s, int64_t e, T need,
                                     unsigned long long &edges)
{
    const int lane = (int)lane_id();
    T found = 0;
    int64_t pos = s;
    while (true) {
        const bool act = need != 0 && found != need && pos < e;
        const unsigned am = __ballot_sync(kFull, act);
        if (!am) break;
        // each open row gets 32 / (open rows) lanes of 4 consecutive slots
        const int per = 32 / __popc(am);
        const int64_t rem = act ? e - pos : 0;
        const int len = (int)(rem < 4 * per ? rem : 4 * per);
        const int nl = (len + 3) >> 2;
        const int incl = warp_inclusive_scan(nl);
        const int excl = incl - nl;
        int o = 0;  // the row this lane serves: the last one starting at or before it
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const int c = o + step;
            if (__shfl_sync(kFull, excl, c) <= lane) o = c;
        }
        const int seg0 = __shfl_sync(kFull, excl, o);
        const int i = lane - seg0;
        const int leno = __shfl_sync(kFull, len, o);
        const int cnt = 4 * i < leno ? (leno - 4 * i < 4 ? leno - 4 * i : 4) : 0;
        const int64_t po = __shfl_sync(kFull, pos, o) + 4 * i;
        const int go = __shfl_sync(kFull, g, o);
        const T need_o = shfl_mask(need, o);
        const T found_o = shfl_mask(found, o);
        const MsGraph &G = s_g[go];
        int32_t c[4];
        T m[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) c[t] = t < cnt ? __ldg(&G.col[po + t]) : -1;
#pragma unroll
        for (int t = 0; t < 4; ++t) m[t] = c[t] >= 0 ? (T)(ld_mask(&M[G.voff + c[t]]) & need_o) : (T)0;
        const T lb = (T)(m[0] | m[1] | m[2] | m[3]);
        // inclusive OR over the earlier lanes of the same row (slot order)
        T x = lb;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const T y = shfl_up_mask(x, d);
            if (lane - d >= seg0) x |= y;
        }
        const T y1 = shfl_up_mask(x, 1);
        const T before = lane > seg0 ? y1 : (T)0;
        T mine = (T)(lb & (T)~before & (T)~found_o);
        const int64_t luo = __shfl_sync(kFull, lu, o);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const T bt = (T)(mine & m[t]);
            if (bt) {
                write_parents(G, S, luo, bt, c[t], true);
                mine &= (T)~bt;
            }
        }
        // each row takes the OR of its slots from its last lane
        const T got = shfl_mask(x, nl > 0 ? incl - 1 : 0);
        if (nl > 0) found |= got;
        pos += len;
        edges += (unsigned long long)len;
    }
    return found;
}

// Warp-collective bottom-up scan of one long row [s, e) of graph g (its vertex
// lu as an original id, for the staged parents) for the bits `need`, 128 entries a round: lane i takes entries
// 4i..4i+3 of the round (one 16-byte load when the columns are aligned) and
// ORs their masks in order; an exclusive prefix-OR over the lanes then gives
// each bit's first supplier in row order (the smallest-id parent), which the
// supplying lane writes.  Stops once every needed bit is found.  Returns the
// bits found (warp-uniform).
template <typename T>
__device__ __forceinline__ T ms_row_warp(const MsGraph *s_g, const MsSlots *S, const T *M, int g,
                                         int64_t lu, int64_t s, int64_t e, T need, bool vec,
                                         unsigned long long &edges)
{
    const int lane = (int)lane_id();
    const MsGraph &G = s_g[g];
    const T *Mg = M + G.voff;
    T found = 0;
    const int64_t s4 = vec ? (s & ~int64_t(3)) : s;
    for (int64_t b = s4; b < e; b += 128) {
        const int64_t p = b + 4 * lane;
        int32_t c[4];
        if (vec) {
            int4 x = make_int4(-1, -1, -1, -1);
            if (p < e) x = __ldg(reinterpret_cast<const int4 *>(G.col + p));
            c[0] = x.x; c[1] = x.y; c[2] = x.z; c[3] = x.w;
        } else {
#pragma unroll
            for (int t = 0; t < 4; ++t) c[t] = p + t < e ? __ldg(&G.col[p + t]) : -1;
        }
        T m[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const bool valid = p + t >= s && p + t < e;
            if (!valid) c[t] = -1;
            m[t] = valid ? (T)(ld_mask(&Mg[c[t]]) & need) : (T)0;
        }
        const T lb = (T)(m[0] | m[1] | m[2] | m[3]);
        // inclusive OR over lanes 0..lane
        T incl = lb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = shfl_up_mask(incl, o);
            if (lane >= o) incl |= y;
        }
        const T up = shfl_up_mask(incl, 1);
        const T before = lane == 0 ? (T)0 : up;
        T mine = (T)(lb & (T)~before & (T)~found);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const T bt = (T)(mine & m[t]);
            if (bt) {
                write_parents(G, S, lu, bt, c[t], true);
                mine &= (T)~bt;
            }
        }
        found |= shfl_mask(incl, 31);
        const int64_t lo = b > s ? b : s, hi = b + 128 < e ? b + 128 : e;
        if (lane == 0) edges += (unsigned long long)(hi - lo);
        if (found == need) break;
    }
    return found;
}

template <typename T>
__global__ void __launch_bounds__(MS_THREADS, 2) ms_kernel(MsArgs<T> a)
{
    __shared__ MsGraph s_g[MS_MAXG];
    __shared__ int64_t s_voff[MS_MAXG + 1];
    __shared__ MsSlots s_slots;
    __shared__ MsWarpBuf s_wb[MS_WARPS];
    __shared__ unsigned long long s_mf, s_any;
    for (int i = threadIdx.x; i < a.ng; i += blockDim.x) s_g[i] = a.graphs[i];
    if (a.slots)
        for (int i = threadIdx.x; i < 64; i += blockDim.x) {
            s_slots.par[i] = a.slots->par[i];
            s_slots.lev[i] = a.slots->lev[i];
            s_slots.start[i] = a.slots->start[i];
        }
    if (threadIdx.x == 0) {
        s_mf = 0;
        s_any = 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= a.ng; i += blockDim.x)
        s_voff[i] = i < a.ng ? s_g[i].voff : s_g[a.ng - 1].voff + s_g[a.ng - 1].n;
    __syncthreads();
    const MsSlots *S = a.slots ? &s_slots : nullptr;
    unsigned bar_target = grid_barrier_base(&a.hdr->bar);
    MsWarpBuf &wb = s_wb[threadIdx.x >> 5];
    int qn_buf = 0, bn_buf = 0;

    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    const unsigned lane = lane_id();
    const int64_t gwarp = gtid >> 5;
    const int64_t nwarps = gthreads >> 5;
    const int64_t ntot = a.ntot;
    const T all = a.do_init
                      ? (a.k >= (int)(8 * sizeof(T)) ? (T)~(T)0 : (T)(((T)1 << a.k) - 1))
                      : (T)a.active;
    MsHeader *h = a.hdr;

    if (a.do_init) {
        // ---- masks clear (the outputs are written once, at the end, from the
        // staged values; a bit is in seen iff its search reached the vertex)
        for (int64_t i = gtid; i < a.mstride; i += gthreads) {
            a.seen[i] = 0;
            a.mbuf[i] = 0;
            a.mbuf[a.mstride + i] = 0;
            a.mbuf[2 * a.mstride + i] = 0;
            if (a.huge && i < ntot && s_g[0].off[i + 1] - s_g[0].off[i] > MS_HUGE)
                a.huge[atomicAdd(&h->nhuge, 1ull)] = (int32_t)i;
        }
        if (!grid_sync(&h->bar, bar_target, a.st, a.timeout_ns, SITE_MS_BAR)) return;
        // roots: bit b of graph g at its root; roots that coincide share one entry
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            unsigned long long na = 0, mf = 0;
            for (int g = 0; g < a.ng; ++g) {
                const MsGraph G = s_g[g];
                for (int b = 0; b < a.k; ++b) {
                    const int64_t r0 = a.roots[(int64_t)g * a.k + b];
                    const int64_t r = G.inv ? (int64_t)G.inv[r0] : r0;
                    const int64_t gid = G.voff + r;
                    if (a.mbuf[gid] == 0) {
                        a.act[na++] = (int32_t)gid;
                        const int64_t deg = G.off[r + 1] - G.off[r];
                        mf += deg;
                        if (deg > MS_BIG_DEG) {
                            const unsigned long long p = h->ctl[0].big;
                            a.bigq[p >> 32] = (unsigned long long)(uint32_t)gid | ((p & 0xffffffffull) << 32);
                            h->ctl[0].big = p + ((1ull << 32) | (unsigned long long)((deg + MS_BIG_CHUNK - 1) / MS_BIG_CHUNK));
                        }
                    }
                    a.mbuf[gid] |= (T)((T)1 << b);
                    a.seen[gid] |= (T)((T)1 << b);
                    a.hist[G.voff + r0] |= (T)((T)1 << b);  // level 0 (staging: original ids)
                    G.pst[r0 * G.kst + b] = (int32_t)r0;
                }
            }
            h->ctl[0].na = na;
            h->ctl[0].mf = mf;
            h->acc[2] = (unsigned long long)a.ng * (unsigned long long)a.k;  // the roots themselves
        }
        if (!grid_sync(&h->bar, bar_target, a.st, a.timeout_ns, SITE_MS_BAR)) return;
    }
    if (a.stats && gtid == 0) h->t0 = globaltimer_ns();

    unsigned long long my_edges = 0, my_touched = 0, reached_new = 0, my_mf = 0;
    T my_any = 0;
    bool prev_td = true;  // the roots' level counts as top-down
    int l = a.l0;
    for (;; ++l) {
        if (a.max_levels > 0 && l >= a.l0 + a.max_levels) break;
        MsCtl *cur = &h->ctl[l % 3];
        const int64_t na = (int64_t)ldcg_u64(&cur->na);
        if (na == 0) break;
        if (l - a.l0 > ntot) {
            if (gtid == 0) record_error(a.st, GB_ERR_TIMEOUT, SITE_MS_LEVELS, l);
            break;
        }
        const int64_t prev_na = l > 0 ? (int64_t)ldcg_u64(&h->na_hist[(l - 1) & 3]) : 0;
        const double mf = (double)ldcg_u64(&cur->mf);
        const unsigned long long bigp = ldcg_u64(&cur->big);
        const int64_t nb = (int64_t)(bigp >> 32), nc = (int64_t)(bigp & 0xffffffffull);
        const bool td = mf * a.ms_alpha < (double)a.nnz_tot && (double)na * a.ms_beta < (double)ntot;
        T *M = a.mbuf + (size_t)(l % 3) * a.mstride;
        T *Mn = a.mbuf + (size_t)((l + 1) % 3) * a.mstride;
        T *Mz = a.mbuf + (size_t)((l + 2) % 3) * a.mstride;
        const int32_t *act = a.act + (size_t)(l % 3) * ntot;
        int32_t *act_next = a.act + (size_t)((l + 1) % 3) * ntot;
        const int32_t *act_prev = a.act + (size_t)((l + 2) % 3) * ntot;
        MsCtl *nxt = &h->ctl[(l + 1) % 3];
        // big-vertex chunk lists alternate between two halves of bigq
        const int64_t bbase = (l & 1) ? a.bigcap : 0;
        unsigned long long *bigq_next = a.bigq + ((l & 1) ? 0 : a.bigcap);

        // Clear the level l-1 frontier (its buffer receives level l+2) and the
        // control record level l+1 will fill; nobody reads either during level l.
        for (int64_t i = gtid; i < prev_na; i += gthreads) Mz[ldcg_i32(&act_prev[i])] = 0;
        if (gtid == 0) {
            MsCtl z = {0, 0, 0, 0};
            h->ctl[(l + 2) % 3] = z;
            h->gnext[(l + 2) & 3] = 0;
        }

        if (td) {
            // (1a) big active vertices in 256-edge chunks
            if (nc > 0) {
                const int64_t per = (nc + nwarps - 1) / nwarps;
                const int64_t c0 = gwarp * per;
                const int64_t c1 = c0 + per < nc ? c0 + per : nc;
                if (c0 < c1) {
                    int64_t lo = 0, hi = nb;
                    while (hi - lo > 1) {
                        const int64_t mid = (lo + hi) >> 1;
                        if ((int64_t)(__ldcg(&a.bigq[bbase + mid]) >> 32) <= c0) lo = mid;
                        else hi = mid;
                    }
                    int64_t ow = lo;
                    unsigned long long be = __ldcg(&a.bigq[bbase + ow]);
                    for (int64_t c = c0; c < c1; ++c) {
                        while (ow + 1 < nb && (int64_t)(__ldcg(&a.bigq[bbase + ow + 1]) >> 32) <= c) {
                            ++ow;
                            be = __ldcg(&a.bigq[bbase + ow]);
                        }
                        const int64_t gv = (int64_t)(uint32_t)(be & 0xffffffffull);
                        const int g = find_graph(s_voff, a.ng, gv);
                        const MsGraph &G = s_g[g];
                        const int64_t lv = gv - G.voff;
                        const T f = ld_mask(&M[gv]);
                        const int64_t s = G.off[lv] + (c - (int64_t)(be >> 32)) * MS_BIG_CHUNK;
                        const int64_t eu = G.off[lv + 1];
                        const int64_t e = s + MS_BIG_CHUNK < eu ? s + MS_BIG_CHUNK : eu;
                        if (lane == 0) my_edges += (unsigned long long)(e - s);
                        for (int64_t b = s; b < e; b += 32) {
                            const int64_t j = b + lane;
                            const bool valid = j < e;
                            const int64_t gu = valid ? G.voff + G.col[j] : 0;
                            ms_td_edge(valid, f, gu, (int32_t)lv, l, a, S, Mn, s_g, s_voff, wb,
                                       qn_buf, bn_buf, my_mf, nxt, act_next, bigq_next);
                        }
                    }
                }
            }
            // (1b) other active vertices, 32 per warp, adjacency gathered as one stream
            for (int64_t i0 = gwarp * 32; i0 < na; i0 += nwarps * 32) {
                const int64_t i = i0 + lane;
                int64_t gv = 0, s = 0, d = 0, vo = 0;
                int g = 0;
                T f = 0;
                if (i < na) {
                    gv = ldcg_i32(&act[i]);
                    g = find_graph(s_voff, a.ng, gv);
                    vo = s_g[g].voff;
                    s = s_g[g].off[gv - vo];
                    d = s_g[g].off[gv - vo + 1] - s;
                    if (d > MS_BIG_DEG) d = 0;
                    f = ld_mask(&M[gv]);
                }
                my_touched += (i < na);
                my_edges += d;
                const int64_t incl = warp_inclusive_scan(d);
                const int64_t total = __shfl_sync(kFull, incl, 31);
                const int64_t excl = incl - d;
                for (int64_t b = 0; b < total; b += 32) {
                    const int64_t kk = b + lane;
                    int owner = 0;
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1) {
                        const int cand = owner + step;
                        if (__shfl_sync(kFull, excl, cand) <= kk) owner = cand;
                    }
                    const int og = __shfl_sync(kFull, g, owner);
                    const int64_t so = __shfl_sync(kFull, s, owner);
                    const int64_t eo = __shfl_sync(kFull, excl, owner);
                    const int64_t vvo = __shfl_sync(kFull, vo, owner);
                    const T fo = shfl_mask(f, owner);
                    const bool valid = kk < total;
                    const int64_t gu = valid ? vvo + s_g[og].col[so + (kk - eo)] : 0;
                    const int32_t pvo = (int32_t)(__shfl_sync(kFull, gv, owner) - vvo);
                    ms_td_edge(valid, fo, gu, pvo, l, a, S, Mn, s_g, s_voff, wb, qn_buf, bn_buf,
                               my_mf, nxt, act_next, bigq_next);
                }
            }
            ms_flush_q(wb, qn_buf, nxt, act_next);
            ms_flush_b(wb, bn_buf, nxt, bigq_next);
            if (!grid_sync(&h->bar, bar_target, a.st, a.timeout_ns, SITE_MS_BAR)) return;
            // (2) the vertices that gained bits join `seen`; in canonical mode
            // each also scans its row for its smallest-id parents and writes
            // its levels (otherwise both were written in (1))
            const int64_t nn = (int64_t)ldcg_u64(&nxt->na);
            for (int64_t i0 = gwarp * 32; i0 < nn; i0 += nwarps * 32) {
                const int64_t i = i0 + lane;
                int64_t gu = 0, lu = 0, rs = 0, re = 0;
                int g = 0;
                T nw = 0;
                if (i < nn) {
                    gu = ldcg_i32(&act_next[i]);
                    g = find_graph(s_voff, a.ng, gu);
                    lu = gu - s_g[g].voff;
                    nw = ld_mask(&Mn[gu]);
                    if (a.canonical) {
                        rs = s_g[g].off[lu];
                        re = s_g[g].off[lu + 1];
                    }
                }
                if (a.canonical) ms_rows(s_g, S, M, g, orig_id(s_g[g], lu), rs, re, nw, my_edges);
                if (i < nn) {
                    if (a.canonical) write_levels(s_g[g], S, lu, nw, l + 1);
                    st_mask(&a.seen[gu], (T)(ld_mask(&a.seen[gu]) | nw));
                    if (a.hist && l + 1 < MS_HIST)
                        a.hist[(size_t)(l + 1) * a.mstride + s_g[g].voff + orig_id(s_g[g], lu)] = nw;
                    reached_new += __popcll((unsigned long long)nw);
                    my_any |= nw;
                }
            }
        } else {
            // bottom-up over all vertices with unseen bits.  First the huge
            // rows (single-graph batches), one per warp, so that the longest
            // scans start at once; then groups of 32 consecutive vertices,
            // handed out by a counter (the next index fetched one group ahead)
            const int64_t nh = a.huge ? (int64_t)ldcg_u64(&h->nhuge) : 0;
            for (int64_t hi = gwarp; hi < nh; hi += nwarps) {
                const int64_t gu = ldcg_i32(&a.huge[hi]);
                const T sn = ld_mask(&a.seen[gu]);
                const T need = all & (T)~sn;
                const int64_t rs = s_g[0].off[gu], re = s_g[0].off[gu + 1];
                T found = 0;
                if (need) {
                    my_touched += (lane == 0);
                    found = ms_row_warp(s_g, S, M, 0, orig_id(s_g[0], gu), rs, re, need, a.vec_col != 0,
                                        my_edges);
                }
                if (found && lane == 0) {
                    write_levels(s_g[0], S, gu, found, l + 1);
                    st_mask(&a.seen[gu], (T)(sn | found));
                    st_mask(&Mn[gu], found);
                    if (a.hist && l + 1 < MS_HIST) a.hist[(size_t)(l + 1) * a.mstride + orig_id(s_g[0], gu)] = found;
                    reached_new += __popcll((unsigned long long)found);
                    my_any |= found;
                }
                ms_append(lane == 0 && found != 0, gu, re - rs, wb, qn_buf, bn_buf, my_mf, nxt, act_next,
                          bigq_next);
            }
            const int64_t ngroups = (ntot + 31) / 32;
            // Only the first bottom-up level after top-down ones, where every
            // row is scanned in full, needs it; later levels keep the static
            // split (cheaper for groups that are mostly done), and so do
            // serving launches (their levels may advance without a launch,
            // which the counter ring does not allow).
            const bool dyn = a.slots == nullptr && prev_td;
            unsigned long long *gctr = &h->gnext[l & 3];
            unsigned long long gnx = dyn ? (lane == 0 ? atomicAdd(gctr, 1ull) : 0ull) : (unsigned long long)gwarp;
            for (;;) {
                const int64_t gi = dyn ? (int64_t)__shfl_sync(kFull, gnx, 0) : (int64_t)gnx;
                if (gi >= ngroups) break;
                if (!dyn) gnx += (unsigned long long)nwarps;
                else if (lane == 0) gnx = atomicAdd(gctr, 1ull);
                const int64_t b0 = gi * 32;
                const int64_t gu = b0 + lane;
                T need = 0;
                int g = 0;
                int64_t lu = 0, deg = 0;
                T sn = 0;
                if (gu < ntot) {
                    sn = ld_mask(&a.seen[gu]);
                    need = all & (T)~sn;
                    if (need) {
                        g = find_graph(s_voff, a.ng, gu);
                        lu = gu - s_g[g].voff;
                        deg = s_g[g].off[lu + 1] - s_g[g].off[lu];
                        if (deg == 0 || (a.huge && deg > MS_HUGE)) need = 0;  // huge: done above
                    }
                }
                int64_t rs = 0, re = 0;
                if (need) {
                    rs = s_g[g].off[lu];
                    re = rs + deg;
                }
                my_touched += (need != 0);
                // the row's original id, loaded once (consecutive rows: one load per warp)
                const T found = ms_rows(s_g, S, M, g, orig_id(s_g[g], lu), rs, re, need, my_edges);
                if (found) {
                    write_levels(s_g[g], S, lu, found, l + 1);
                    st_mask(&a.seen[gu], (T)(sn | found));
                    st_mask(&Mn[gu], found);
                    if (a.hist && l + 1 < MS_HIST)
                        a.hist[(size_t)(l + 1) * a.mstride + s_g[g].voff + orig_id(s_g[g], lu)] = found;
                    reached_new += __popcll((unsigned long long)found);
                    my_any |= found;
                }
                ms_append(found != 0, gu, deg, wb, qn_buf, bn_buf, my_mf, nxt, act_next, bigq_next);
            }
            ms_flush_q(wb, qn_buf, nxt, act_next);
            ms_flush_b(wb, bn_buf, nxt, bigq_next);
        }
        // end of level: the block's degree sum and advancing bits, one atomic each
        {
            const unsigned long long t = warp_sum(my_mf);
            const unsigned long long o = (unsigned long long)warp_or(my_any);
            my_mf = 0;
            my_any = 0;
            if (lane == 0) {
                if (t) atomicAdd(&s_mf, t);
                if (o) atomicOr(&s_any, o);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                if (s_mf) atomicAdd(&nxt->mf, s_mf);
                if (s_any) atomicOr(&nxt->anynew, s_any);
                s_mf = 0;
                s_any = 0;
            }
        }
        prev_td = td;
        if (gtid == 0) {
            h->na_hist[l & 3] = (unsigned long long)na;
            atomicAdd(&h->acc[td ? 4 : 5], 1ull);
        }
        if (!grid_sync(&h->bar, bar_target, a.st, a.timeout_ns, SITE_MS_BAR)) return;
        // per-level device time, active vertices and step
        if (a.stats && gtid == 0 && l - a.l0 < kStatLevels) {
            const uint64_t now = globaltimer_ns();
            a.stats->level_ns[l - a.l0] = now - h->t0;
            a.stats->level_frontier[l - a.l0] = na;
            a.stats->level_dir[l - a.l0] = td ? 1 : 2;
            h->t0 = now;
        }
    }

    // ---- batch calls: the [k][n] outputs from the staged values, each entry
    // written once; a warp takes 32 consecutive vertices, so for every bit the
    // warp's stores fill one contiguous run of the output row
    if (!a.slots) {
        for (int64_t v0 = gwarp * 32; v0 < ntot; v0 += nwarps * 32) {
            const int64_t gv = v0 + lane;
            if (gv >= ntot) continue;
            const int g = find_graph(s_voff, a.ng, gv);
            const MsGraph &G = s_g[g];
            const int64_t lu = gv - G.voff;  // the output's vertex (original id)
            // the reached bits from the search state (by search id); the
            // staged parents, levels and level masks are by original id
            const T sn = ld_mask(&a.seen[G.voff + (G.inv ? (int64_t)G.inv[lu] : lu)]);
            T hm[MS_HIST];
#pragma unroll
            for (int j = 0; j < MS_HIST; ++j) hm[j] = a.hist[(size_t)j * a.mstride + gv];
            if ((G.kst & 15) == 0) {
                // the vertex's staged parents 16 at a time, as four 16-byte loads
                const int4 *prow = reinterpret_cast<const int4 *>(G.pst + lu * G.kst);
                for (int b0 = 0; b0 < a.k; b0 += 16) {
                    int32_t pv[16];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int4 x = prow[(b0 >> 2) + q];
                        pv[4 * q] = x.x;
                        pv[4 * q + 1] = x.y;
                        pv[4 * q + 2] = x.z;
                        pv[4 * q + 3] = x.w;
                    }
#pragma unroll
                    for (int t = 0; t < 16; ++t) {
                        const int b = b0 + t;
                        if (b >= a.k) break;
                        const bool has = (sn >> b) & 1;
                        int32_t lvl = -1;
#pragma unroll
                        for (int j = 0; j < MS_HIST; ++j)
                            if ((hm[j] >> b) & 1) lvl = j;
                        if (has && lvl < 0) lvl = G.lst[lu * G.kst + b];
                        G.par[(int64_t)b * G.n + lu] = has ? pv[t] : -1;
                        G.lev[(int64_t)b * G.n + lu] = has ? lvl : -1;
                    }
                }
            } else {
                for (int b = 0; b < a.k; ++b) {
                    const bool has = (sn >> b) & 1;
                    int32_t lvl = -1;
#pragma unroll
                    for (int j = 0; j < MS_HIST; ++j)
                        if ((hm[j] >> b) & 1) lvl = j;
                    if (has && lvl < 0) lvl = G.lst[lu * G.kst + b];
                    G.par[(int64_t)b * G.n + lu] = has ? G.pst[lu * G.kst + b] : -1;
                    G.lev[(int64_t)b * G.n + lu] = has ? lvl : -1;
                }
            }
        }
    }

    if (!a.stats) return;
    my_edges = warp_sum(my_edges);
    my_touched = warp_sum(my_touched);
    reached_new = warp_sum(reached_new);
    if (lane == 0) {
        if (my_edges) atomicAdd(&h->acc[0], my_edges);
        if (my_touched) atomicAdd(&h->acc[1], my_touched);
        if (reached_new) atomicAdd(&h->acc[2], reached_new);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&h->done, 1u);
        if (prev == gridDim.x - 1) {
            __threadfence();
            BfsDevStats &st = *a.stats;
            st.nlevels = (unsigned long long)l;
            st.edges_examined = ldcg_u64(&h->acc[0]);
            st.vertices_touched = ldcg_u64(&h->acc[1]);
            st.reached = ldcg_u64(&h->acc[2]);
            st.td_levels = ldcg_u64(&h->acc[4]);
            st.bu_levels = ldcg_u64(&h->acc[5]);
        }
    }
}

template <typename T>
gb_status ms_launch(std::vector<MsGraph> gs, int k, const std::vector<int64_t> &roots,
                    int64_t nnz_tot, BfsDevStats *stats, cudaStream_t s)
{
    Context *ctx = context();
    if (!ctx) return GB_ERR_CUDA;
    const gb_bfs_options &o = options();
    const int ng = (int)gs.size();
    int64_t ntot = 0;
    for (int i = 0; i < ng; ++i) {
        gs[i].voff = ntot;
        ntot += gs[i].n;
    }
    if (ntot >= (int64_t(1) << 31)) {
        set_error("multi-source BFS: more than 2^31 vertices in total");
        return GB_ERR_RANGE;
    }
    // Byte masks are updated with 32-bit atomics, so every mask array is padded.
    const int64_t np = (ntot + 63) & ~int64_t(63);
    const int64_t bigcap = nnz_tot / (MS_BIG_DEG + 1) + ng * k + 2;
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t o_g = up(sizeof(MsHeader));
    const size_t o_r = o_g + up(ng * sizeof(MsGraph));
    const size_t o_seen = o_r + up((size_t)ng * k * sizeof(int64_t));
    const size_t o_m = o_seen + up(np * sizeof(T));
    const size_t o_act = o_m + up(3 * np * sizeof(T));
    const size_t o_big = o_act + up(3 * (size_t)ntot * sizeof(int32_t));
    const size_t o_huge = o_big + up(2 * bigcap * sizeof(unsigned long long));
    const int64_t hugecap = ng == 1 ? nnz_tot / (MS_HUGE + 1) + 1 : 0;
    const size_t total = o_huge + hugecap * sizeof(int32_t);
    unsigned char *ws = nullptr;
    Scratch tmp(s);
    GB_CUDA(tmp.alloc(&ws, total));
    // vertex-major staging of parents and levels, [ntot][k] each
    int32_t *stage = nullptr;
    GB_CUDA(tmp.alloc(&stage, 2 * (size_t)ntot * k));
    T *hist = nullptr;  // reached-bit masks of the first MS_HIST levels
    GB_CUDA(tmp.alloc(&hist, (size_t)MS_HIST * np));
    GB_CUDA(cudaMemsetAsync(hist, 0, (size_t)MS_HIST * np * sizeof(T), s));
    for (int i = 0; i < ng; ++i) {
        gs[i].pst = stage + gs[i].voff * k;
        gs[i].lst = stage + (size_t)ntot * k + gs[i].voff * k;
        gs[i].kst = k;
    }
    GB_CUDA(cudaMemsetAsync(ws, 0, sizeof(MsHeader), s));
    GB_CUDA(cudaMemcpyAsync(ws + o_g, gs.data(), ng * sizeof(MsGraph), cudaMemcpyHostToDevice, s));
    GB_CUDA(cudaMemcpyAsync(ws + o_r, roots.data(), (size_t)ng * k * sizeof(int64_t),
                            cudaMemcpyHostToDevice, s));
    MsArgs<T> a;
    a.graphs = reinterpret_cast<const MsGraph *>(ws + o_g);
    a.ng = ng;
    a.k = k;
    a.ntot = ntot;
    a.mstride = np;
    a.nnz_tot = nnz_tot;
    a.roots = reinterpret_cast<const int64_t *>(ws + o_r);
    a.seen = reinterpret_cast<T *>(ws + o_seen);
    a.mbuf = reinterpret_cast<T *>(ws + o_m);
    a.hist = hist;
    a.act = reinterpret_cast<int32_t *>(ws + o_act);
    a.bigq = reinterpret_cast<unsigned long long *>(ws + o_big);
    a.bigcap = bigcap;
    a.hdr = reinterpret_cast<MsHeader *>(ws);
    a.st = ctx->status;
    a.stats = stats;
    a.ms_alpha = (float)o.ms_alpha;
    a.ms_beta = (float)o.ms_beta;
    a.timeout_ns = timeout_ns();
    a.canonical = o.canonical_parents;
    a.l0 = 0;
    a.max_levels = 0;
    a.do_init = 1;
    a.active = 0;
    a.slots = nullptr;
    a.huge = hugecap ? reinterpret_cast<int32_t *>(ws + o_huge) : nullptr;
    a.vec_col = 1;
    for (int i = 0; i < ng; ++i)
        if (reinterpret_cast<uintptr_t>(gs[i].col) & 15u) a.vec_col = 0;
    void *args[] = {&a};
    GB_CUDA(cudaLaunchCooperativeKernel((const void *)ms_kernel<T>, dim3(ctx->ms_blocks),
                                        dim3(MS_THREADS), args, 0, s));
    note_launch();
    return GB_OK;
}

// Serialises the build of a graph's degree-ordered copy by batched calls.
std::mutex g_layout_mu;

}  // namespace

gb_status prepare_batched(gb_graph *g, cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(g_layout_mu);
    return build_batched_layout(g, s);
}

gb_status msbfs_impl(const gb_graph *g, const int64_t *roots, int k, int32_t *parents,
                     int32_t *levels, BfsDevStats *stats, cudaStream_t s)
{
    // A graph whose frontier masks (8 n bytes) outgrow the L2 is searched on its
    // degree-ordered copy, built at the first batched call if not yet there.
    if (!g->rl_col && g->n >= MS_LAYOUT_MIN_N) {
        gb_status rc = prepare_batched(const_cast<gb_graph *>(g), s);
        if (rc != GB_OK) return rc;
    }
    MsGraph G;
    G.off = g->rl_col ? g->rl_off : g->off;
    G.col = g->rl_col ? g->rl_col : g->col;
    G.perm = g->rl_col ? g->rl_perm : nullptr;
    G.inv = g->rl_col ? g->rl_inv : nullptr;
    G.nz = g->nz;
    G.voff = 0;
    G.n = g->n;
    G.par = parents;
    G.lev = levels;
    std::vector<int64_t> r(roots, roots + k);
    return ms_launch<unsigned long long>({G}, k, r, g->nnz, stats, s);
}

gb_status multigraph_impl(const gb_graph *const *gs, int ng, const int64_t *roots, int r,
                          int32_t *const *parents, int32_t *const *levels, BfsDevStats *stats,
                          cudaStream_t s)
{
    std::vector<MsGraph> v(ng);
    int64_t nnz = 0;
    for (int i = 0; i < ng; ++i) {
        v[i].off = gs[i]->off;
        v[i].col = gs[i]->col;
        v[i].nz = gs[i]->nz;
        v[i].perm = nullptr;
        v[i].inv = nullptr;
        v[i].voff = 0;
        v[i].n = gs[i]->n;
        v[i].par = parents[i];
        v[i].lev = levels[i];
        nnz += gs[i]->nnz;
    }
    std::vector<int64_t> rr(roots, roots + (size_t)ng * r);
    return ms_launch<unsigned char>(v, r, rr, nnz, stats, s);
}

// ---------------------------------------------------------------------------
// Serving: a resident graph's search state, admissions and one-level steps.
// ---------------------------------------------------------------------------
namespace {

// seen[u] loses the bits `fresh` (slots being reused), except that isolated
// vertices keep them set: no query reaches them and bottom-up skips them.
__global__ void ms_admit_clear_kernel(const uint32_t *__restrict__ nz, int64_t n,
                                      unsigned long long *__restrict__ seen,
                                      unsigned long long fresh)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        const bool iso = !((nz[u >> 5] >> (u & 31)) & 1u);
        seen[u] = (seen[u] & ~fresh) | (iso ? fresh : 0ull);
    }
}

struct AdmitList {
    int count;
    int level;
    int bit[64];
    int64_t root[64];
    int32_t *par[64];
    int32_t *lev[64];
};

// One thread: place each admitted root into level l's frontier.
__global__ void ms_admit_roots_kernel(MsGraph G, MsHeader *h, unsigned long long *seen,
                                      unsigned long long *Ml, int32_t *act_l,
                                      unsigned long long *bigq_l, int l, AdmitList adm,
                                      MsSlots *slots)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    MsCtl &c = h->ctl[l % 3];
    for (int i = 0; i < adm.count; ++i) {
        const int b = adm.bit[i];
        const int64_t r = adm.root[i];
        const unsigned long long bit = 1ull << b;
        // the slot table entry travels in the kernel parameters: no host copy
        slots->par[b] = adm.par[i];
        slots->lev[b] = adm.lev[i];
        slots->start[b] = adm.level;
        seen[r] |= bit;
        if (Ml[r] == 0) {
            act_l[c.na++] = (int32_t)r;
            const int64_t deg = G.off[r + 1] - G.off[r];
            c.mf += (unsigned long long)deg;
            if (deg > MS_BIG_DEG) {
                const unsigned long long p = c.big;
                bigq_l[p >> 32] = (unsigned long long)(uint32_t)r | ((p & 0xffffffffull) << 32);
                c.big = p + ((1ull << 32) | (unsigned long long)((deg + MS_BIG_CHUNK - 1) / MS_BIG_CHUNK));
            }
        }
        Ml[r] |= bit;
        slots->lev[b][r] = 0;
        slots->par[b][r] = (int32_t)r;
    }
}

}  // namespace

struct MsServe {
    const gb_graph *g = nullptr;
    unsigned char *ws = nullptr;
    MsHeader *hdr = nullptr;
    MsGraph *graph_dev = nullptr;
    MsSlots *slots_dev = nullptr;
    unsigned long long *seen = nullptr;
    unsigned long long *mbuf = nullptr;
    int32_t *act = nullptr;
    unsigned long long *bigq = nullptr;
    int64_t bigcap = 0;
    int64_t mstride = 0;
    int blocks = 0;
    size_t ws_bytes = 0;
    MsGraph graph_host;
};

gb_status ms_serve_create(const gb_graph *g, int blocks, MsServe **out, cudaStream_t s)
{
    Context *ctx = context();
    if (!ctx) return GB_ERR_CUDA;
    MsServe *m = new MsServe();
    m->g = g;
    const int64_t n = g->n;
    m->mstride = (n + 63) & ~int64_t(63);
    m->bigcap = g->nnz / (MS_BIG_DEG + 1) + 66;
    m->blocks = std::max(1, std::min(blocks, ctx->ms_blocks));
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t o_g = up(sizeof(MsHeader));
    const size_t o_sl = o_g + up(sizeof(MsGraph));
    const size_t o_seen = o_sl + up(sizeof(MsSlots));
    const size_t o_m = o_seen + up(m->mstride * 8);
    const size_t o_act = o_m + up(3 * m->mstride * 8);
    const size_t o_big = o_act + up(3 * (size_t)n * 4);
    const size_t total = o_big + 2 * m->bigcap * 8;
    m->ws_bytes = total;
    cudaError_t e = gb::dmalloc((void **)&m->ws, total);
    if (e != cudaSuccess) {
        delete m;
        return cuda_fail(e, "server workspace");
    }
    m->hdr = reinterpret_cast<MsHeader *>(m->ws);
    m->graph_dev = reinterpret_cast<MsGraph *>(m->ws + o_g);
    m->slots_dev = reinterpret_cast<MsSlots *>(m->ws + o_sl);
    m->seen = reinterpret_cast<unsigned long long *>(m->ws + o_seen);
    m->mbuf = reinterpret_cast<unsigned long long *>(m->ws + o_m);
    m->act = reinterpret_cast<int32_t *>(m->ws + o_act);
    m->bigq = reinterpret_cast<unsigned long long *>(m->ws + o_big);
    MsGraph G;
    G.off = g->off;
    G.col = g->col;
    G.nz = g->nz;
    G.perm = nullptr;  // serving searches the graph itself
    G.inv = nullptr;
    G.voff = 0;
    G.n = n;
    G.par = nullptr;
    G.lev = nullptr;
    G.pst = nullptr;  // serving writes into the per-query slots instead
    G.lst = nullptr;
    G.kst = 0;
    m->graph_host = G;
    if ((e = cudaMemsetAsync(m->ws, 0, o_big, s)) == cudaSuccess &&
        (e = cudaMemcpyAsync(m->graph_dev, &m->graph_host, sizeof(MsGraph), cudaMemcpyHostToDevice, s)) ==
            cudaSuccess) {
        ms_admit_clear_kernel<<<ctx->num_sms * 4, 256, 0, s>>>(g->nz, n, m->seen, ~0ull);
        note_launch();
        if ((e = cudaGetLastError()) == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) {
        gb::dfree(m->ws);
        delete m;
        return cuda_fail(e, "server workspace");
    }
    *out = m;
    return GB_OK;
}

size_t ms_serve_bytes(const MsServe *m) { return m ? m->ws_bytes : 0; }

void ms_serve_destroy(MsServe *m)
{
    if (!m) return;
    if (m->ws) gb::dfree(m->ws);
    delete m;
}

gb_status ms_serve_admit(MsServe *m, int level, int count, const int *bits, const int64_t *roots,
                         const MsSlots *table, cudaStream_t s)
{
    Context *ctx = context();
    if (!ctx) return GB_ERR_CUDA;
    if (count < 1 || count > 64) return GB_OK;
    AdmitList adm;
    adm.count = count;
    adm.level = level;
    unsigned long long fresh = 0;
    for (int i = 0; i < count; ++i) {
        adm.bit[i] = bits[i];
        adm.root[i] = roots[i];
        adm.par[i] = table->par[bits[i]];
        adm.lev[i] = table->lev[bits[i]];
        fresh |= 1ull << bits[i];
    }
    ms_admit_clear_kernel<<<ctx->num_sms * 4, 256, 0, s>>>(m->g->nz, m->g->n, m->seen, fresh);
    note_launch();
    const int64_t ntot = m->g->n;
    ms_admit_roots_kernel<<<1, 32, 0, s>>>(m->graph_host, m->hdr, m->seen,
                                           m->mbuf + (size_t)(level % 3) * m->mstride,
                                           m->act + (size_t)(level % 3) * ntot,
                                           m->bigq + ((level & 1) ? m->bigcap : 0), level, adm,
                                           m->slots_dev);
    note_launch();
    GB_CUDA(cudaGetLastError());
    return GB_OK;
}

gb_status ms_serve_step(MsServe *m, int level, unsigned long long active, MsCtl *host_ctl,
                        cudaStream_t s)
{
    Context *ctx = context();
    if (!ctx) return GB_ERR_CUDA;
    const gb_bfs_options &o = options();
    MsArgs<unsigned long long> a;
    a.graphs = m->graph_dev;
    a.ng = 1;
    a.k = 64;
    a.ntot = m->g->n;
    a.mstride = m->mstride;
    a.nnz_tot = m->g->nnz;
    a.roots = nullptr;
    a.seen = m->seen;
    a.mbuf = m->mbuf;
    a.hist = nullptr;  // serving writes levels into the per-query slots
    a.act = m->act;
    a.bigq = m->bigq;
    a.bigcap = m->bigcap;
    a.hdr = m->hdr;
    a.st = ctx->status;
    a.stats = nullptr;
    a.ms_alpha = (float)o.ms_alpha;
    a.ms_beta = (float)o.ms_beta;
    a.timeout_ns = timeout_ns();
    a.canonical = o.canonical_parents;
    a.l0 = level;
    a.max_levels = 1;
    a.do_init = 0;
    a.active = active;
    a.slots = m->slots_dev;
    a.vec_col = (reinterpret_cast<uintptr_t>(m->g->col) & 15u) == 0;
    a.huge = nullptr;
    void *args[] = {&a};
    GB_CUDA(cudaLaunchCooperativeKernel((const void *)ms_kernel<unsigned long long>, dim3(m->blocks),
                                        dim3(MS_THREADS), args, 0, s));
    note_launch();
    GB_CUDA(cudaMemcpyAsync(host_ctl, &m->hdr->ctl[(level + 1) % 3], sizeof(MsCtl),
                            cudaMemcpyDeviceToHost, s));
    return GB_OK;
}

int msbfs_pick_blocks(int num_sms)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ms_kernel<unsigned long long>,
                                                      MS_THREADS, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    int per_sm8 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm8, ms_kernel<unsigned char>,
                                                      MS_THREADS, 0) != cudaSuccess ||
        per_sm8 < 1)
        per_sm8 = 1;
    return num_sms * std::min(std::min(per_sm, per_sm8), 2);
}

}  // namespace gb
