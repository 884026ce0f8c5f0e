// Kernel 1 (Sec. 2.2): the undirected CSR graph from the Kronecker tuples.
//
//   1. symmetrise: tuple (u,v) becomes keys (u << S | v) and (v << S | u),
//      S = scale, so one key holds an ordered pair in 2*S contiguous bits;
//   2. radix sort of the keys (ceil(2S/8) passes): the CSR of Sec. 2.2 is
//      built from the edges in sorted order (Sec. 4.2: by a parallel sort);
//   3. a key is kept if it is not a self-loop (u == v) and differs from its
//      predecessor (a duplicate; Sec. 2.1 lets later kernels drop both); a count pass and a
//      scan of the per-tile counts give each kept key its column slot;
//   4. the write pass stores the columns and, at every change of row between
//      neighbouring keys, the offsets of all rows in between: an empty row
//      repeats the previous offset and off[n] = nnz (Sec. 2.2).
//
// Two per-vertex arrays that the search consults are derived from the CSR:
// the degree >= 1 bitmap, and for every row one of its neighbours of largest
// degree (the "hub" that the bottom-up step tests first: a neighbour with many
// edges is the likeliest to sit in the frontier; rows longer than HUB_SCAN
// are sampled by their first HUB_SCAN entries).
#include "common.cuh"
#include "internal.h"

#include <algorithm>

namespace gb {
namespace {

constexpr int FIN_THREADS = 256;
constexpr int FIN_ITEMS = 16;
constexpr int FIN_TILE = FIN_THREADS * FIN_ITEMS;  // 4096 keys
constexpr int SITE_K1_RANGE = 10;

// Both directed keys of every tuple, and the digit counts of the radix
// sort's passes over them (plan.passes of them; 0: none), so that the sort
// does not read the keys once more for its histogram.
constexpr int SYM_THREADS = 256;
__global__ void __launch_bounds__(SYM_THREADS) k1_sym_kernel(const int64_t *__restrict__ edges, int64_t m,
                                                             int scale, ulonglong2 *__restrict__ keys,
                                                             SortPlan plan, unsigned long long *__restrict__ hist,
                                                             DevStatus *st)
{
    __shared__ unsigned s_h[RS_MAX_PASSES][RS_RADIX_MAX];
    const int passes = plan.passes;
    for (int i = threadIdx.x; i < RS_MAX_PASSES * RS_RADIX_MAX; i += blockDim.x) (&s_h[0][0])[i] = 0;
    __syncthreads();
    const int64_t n = int64_t(1) << scale;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        int64_t u = edges[e];
        int64_t v = edges[m + e];
        if (u < 0 || u >= n || v < 0 || v >= n) {
            record_error(st, GB_ERR_RANGE, SITE_K1_RANGE, (long long)e);
            u = v = 0;  // a self-loop: dropped below
        }
        const uint64_t ka = ((uint64_t)u << scale) | (uint64_t)v;
        const uint64_t kb = ((uint64_t)v << scale) | (uint64_t)u;
        keys[e] = make_ulonglong2(ka, kb);
#pragma unroll
        for (int q = 0; q < RS_MAX_PASSES; ++q) {  // unrolled: the plan stays in registers
            if (q >= passes) break;
            const unsigned dm = (1u << plan.bits[q]) - 1u;
            atomicAdd(&s_h[q][(unsigned)(ka >> plan.shift[q]) & dm], 1u);
            atomicAdd(&s_h[q][(unsigned)(kb >> plan.shift[q]) & dm], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * RS_RADIX_MAX; i += blockDim.x) {
        const unsigned c = (&s_h[0][0])[i];
        if (c) atomicAdd(&hist[i], (unsigned long long)c);
    }
}

__device__ __forceinline__ bool k1_keep(const uint64_t *keys, int64_t i, uint64_t k, int scale,
                                        uint64_t vmask)
{
    if ((k >> scale) == (k & vmask)) return false;  // self-loop
    return i == 0 || keys[i - 1] != k;              // first of a run of duplicates
}

// Warp w of a tile takes keys [t0 + w*WARP_KEYS, +WARP_KEYS) here and in the
// write pass; the kept keys are counted per warp and per tile.
constexpr int FIN_WARPS = FIN_THREADS / 32;
constexpr int WARP_KEYS = FIN_TILE / FIN_WARPS;  // 512
__global__ void __launch_bounds__(FIN_THREADS) k1_count_kernel(const uint64_t *__restrict__ keys,
                                                               int64_t nk, int scale,
                                                               unsigned *__restrict__ tile_cnt,
                                                               unsigned *__restrict__ warp_cnt)
{
    __shared__ unsigned s_w[FIN_WARPS];
    const uint64_t vmask = (uint64_t(1) << scale) - 1;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t w0 = (int64_t)blockIdx.x * FIN_TILE + (int64_t)warp * WARP_KEYS;
    unsigned c = 0;
#pragma unroll 4
    for (int j = 0; j < WARP_KEYS / 32; ++j) {
        const int64_t i = w0 + 32 * j + lane;
        if (i < nk) c += k1_keep(keys, i, keys[i], scale, vmask);
    }
    c = warp_sum(c);
    if (lane == 0) {
        s_w[warp] = c;
        warp_cnt[(int64_t)blockIdx.x * FIN_WARPS + warp] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int w = 0; w < FIN_THREADS / 32; ++w) t += s_w[w];
        tile_cnt[blockIdx.x] = t;
    }
}

// Exclusive scan of the tile counts (one block; each thread a contiguous run).
__global__ void __launch_bounds__(1024) k1_scan_tiles_kernel(const unsigned *__restrict__ cnt,
                                                             int64_t ntiles,
                                                             unsigned long long *__restrict__ base)
{
    __shared__ unsigned long long s_w[32];
    const int tid = threadIdx.x;
    const int64_t per = (ntiles + blockDim.x - 1) / blockDim.x;
    const int64_t b0 = (int64_t)tid * per;
    const int64_t b = b0 < ntiles ? b0 : ntiles;
    const int64_t e = b + per < ntiles ? b + per : ntiles;
    unsigned long long sum = 0;
    for (int64_t i = b; i < e; ++i) sum += cnt[i];
    unsigned long long incl = warp_inclusive_scan(sum);
    if ((tid & 31) == 31) s_w[tid >> 5] = incl;
    __syncthreads();
    if (tid < 32) {
        unsigned long long w = s_w[tid];
        unsigned long long wi = warp_inclusive_scan(w);
        s_w[tid] = wi - w;
    }
    __syncthreads();
    unsigned long long run = s_w[tid >> 5] + incl - sum;
    for (int64_t i = b; i < e; ++i) {
        base[i] = run;
        run += cnt[i];
    }
    if (tid == blockDim.x - 1) base[ntiles] = run;
}

// Warp-striped like the count: lane i of round j takes the key
// t0 + w*WARP_KEYS + 32 j + i, so that loads and column stores are
// coalesced; a key's predecessor comes from the next-lower lane (lane 0: the
// previous round's lane 31, or memory at the warp's start).  The warp's first
// column position (the tile's base plus the counts of the tile's earlier
// warps) is loaded together with its keys: one pass, no block barrier.
__global__ void __launch_bounds__(FIN_THREADS) k1_write_kernel(
    const uint64_t *__restrict__ keys, int64_t nk, int scale,
    const unsigned long long *__restrict__ tile_base, const unsigned *__restrict__ warp_cnt,
    int64_t n, int64_t *__restrict__ off, int32_t *__restrict__ col, int64_t nnz, DevStatus *st)
{
    const uint64_t vmask = (uint64_t(1) << scale) - 1;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t w0 = (int64_t)blockIdx.x * FIN_TILE + (int64_t)warp * WARP_KEYS;
    constexpr int ROUNDS = WARP_KEYS / 32;
    const unsigned wc = lane < warp ? warp_cnt[(int64_t)blockIdx.x * FIN_WARPS + lane] : 0u;
    const unsigned long long tb = tile_base[blockIdx.x];
    uint64_t k[ROUNDS];
#pragma unroll
    for (int j = 0; j < ROUNDS; ++j) {
        const int64_t i = w0 + 32 * j + lane;
        k[j] = i < nk ? keys[i] : 0;
    }
    uint64_t prev = w0 > 0 && w0 - 1 < nk ? keys[w0 - 1] : ~0ull;  // predecessor of the warp's first key
    int64_t base = (int64_t)tb + (int64_t)warp_sum(wc);
    // columns at their positions (self-loops and repeats dropped); every
    // change of row writes the offsets of the rows it passes (an empty row
    // repeats the offset)
#pragma unroll
    for (int j = 0; j < ROUNDS; ++j) {
        const int64_t i = w0 + 32 * j + lane;
        uint64_t kp = __shfl_up_sync(kFull, k[j], 1);
        if (lane == 0) kp = prev;
        prev = __shfl_sync(kFull, k[j], 31);
        const bool keep = i < nk && (k[j] >> scale) != (k[j] & vmask) && (i == 0 || kp != k[j]);
        const unsigned keepm = __ballot_sync(kFull, keep);
        const int64_t pos = base + __popc(keepm & lanemask_lt());
        if (i < nk) {
            const int64_t r = (int64_t)(k[j] >> scale);
            const int64_t rp = i == 0 ? -1 : (int64_t)(kp >> scale);
            for (int64_t x = rp + 1; x <= r; ++x) off[x] = pos;  // rows rp+1..r start here
            if (keep) {
                if (pos < nnz) col[pos] = (int32_t)(k[j] & vmask);
                else record_error(st, GB_ERR_RANGE, 11, pos);
            }
            if (i == nk - 1) {
                const int64_t end = pos + (keep ? 1 : 0);
                for (int64_t x = r + 1; x <= n; ++x) off[x] = end;  // trailing empty rows, off[n]
            }
        }
        base += __popc(keepm);
    }
}

// Bit v of word v/32: row v is not empty.  One warp per word.
__global__ void nz_bitmap_kernel(const int64_t *__restrict__ off, int64_t n,
                                 uint32_t *__restrict__ nz, int64_t nw)
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

// The list of vertices of degree >= 1 in ascending order (the first
// bottom-up level of a search walks it instead of the whole visited bitmap):
// per block of NZL_WORDS bitmap words a count, a scan of the counts, then
// each block writes its vertices.
constexpr int NZL_WORDS = 1024;

__global__ void __launch_bounds__(NZL_WORDS) nzl_count_kernel(const uint32_t *__restrict__ nz, int64_t nw,
                                                             unsigned *__restrict__ cnt)
{
    __shared__ unsigned s_w[NZL_WORDS / 32];
    const int64_t w = (int64_t)blockIdx.x * NZL_WORDS + threadIdx.x;
    const unsigned c = warp_sum(w < nw ? (unsigned)__popc(nz[w]) : 0u);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
        const unsigned t = warp_sum(s_w[threadIdx.x]);
        if (threadIdx.x == 0) cnt[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(NZL_WORDS) nzl_write_kernel(const uint32_t *__restrict__ nz, int64_t nw,
                                                             const unsigned long long *__restrict__ base,
                                                             int32_t *__restrict__ list)
{
    __shared__ unsigned s_w[NZL_WORDS / 32];
    const int64_t w = (int64_t)blockIdx.x * NZL_WORDS + threadIdx.x;
    unsigned bits = w < nw ? nz[w] : 0u;
    const unsigned c = (unsigned)__popc(bits);
    const unsigned incl = warp_inclusive_scan(c);
    if ((threadIdx.x & 31) == 31) s_w[threadIdx.x >> 5] = incl;
    __syncthreads();
    unsigned long long pos = base[blockIdx.x] + incl - c;
    for (int k = 0; k < (int)(threadIdx.x >> 5); ++k) pos += s_w[k];
    while (bits) {
        const int b = __ffs(bits) - 1;
        bits &= bits - 1;
        list[pos++] = (int32_t)(w * 32 + b);
    }
}

// hd[v] = (hub[v], min(degree(v), 65535)): the bottom-up list walks read both
// with one 8-byte load instead of a hub load and two 8-byte offsets from
// other sectors.
__global__ void hd_kernel(const int64_t *__restrict__ off, const int32_t *__restrict__ hub, int64_t n,
                          int2 *__restrict__ hd)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t d = off[v + 1] - off[v];
        hd[v] = make_int2(hub[v], (int)(d < 65535 ? d : 65535));
    }
}

constexpr int HUB_THREADS = 256;
constexpr int64_t HUB_SCAN = 128;  // entries of a row examined for its hub

// An 8-bit increasing key of the degree: 8 * floor(log2 d) + the next three
// bits of d, plus one (0 for an empty row).
__global__ void deg_key_kernel(const int64_t *__restrict__ off, int64_t n, uint8_t *__restrict__ key)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t d = off[v + 1] - off[v];
        unsigned k = 0;
        if (d > 0) {
            const int e = 63 - __clzll(d);
            const unsigned m = e >= 3 ? (unsigned)(d >> (e - 3)) & 7u : (unsigned)(d << (3 - e)) & 7u;
            k = (unsigned)e * 8u + m + 1u;
            if (k > 255u) k = 255u;
        }
        key[v] = (uint8_t)k;
    }
}

// hub[u] = among the first HUB_SCAN neighbours of u (all of them for a shorter
// row) the one with the largest degree key, the smallest id among equals; -1
// for an empty row.  The hub is a heuristic (the bottom-up step tests it
// first), so long rows, whose vertices are reached early anyway, are only
// sampled: every row costs at most HUB_SCAN entries.  A warp
// takes 32 rows and streams their edges as one sequence (lane k of a round
// reads entry k), each edge folded into its row's slot with a shared-memory
// atomic max of (key << 32 | ~v).
__global__ void __launch_bounds__(HUB_THREADS) hub_kernel(const int64_t *__restrict__ off,
                                                          const int32_t *__restrict__ col,
                                                          const uint8_t *__restrict__ key, int64_t n,
                                                          int64_t nnz, int32_t *__restrict__ hub,
                                                          DevStatus *st)
{
    __shared__ unsigned long long s_best[HUB_THREADS];
    const unsigned lane = threadIdx.x & 31u;
    const int wbase = threadIdx.x & ~31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r0 = gwarp * 32; r0 < n; r0 += nwarps * 32) {
        const int64_t r = r0 + lane;
        int64_t s0 = 0, d = 0;
        if (r < n) {
            s0 = off[r];
            d = off[r + 1] - s0;
            if (d < 0 || s0 < 0 || s0 + d > nnz) d = 0;
            if (d > HUB_SCAN) d = HUB_SCAN;
        }
        s_best[threadIdx.x] = 0;
        __syncwarp();
        const int64_t incl = warp_inclusive_scan(d);
        const int64_t total = __shfl_sync(kFull, incl, 31);
        const int64_t excl = incl - d;
        for (int64_t b = 0; b < total; b += 32) {
            const int64_t k = b + lane;
            int owner = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int cand = owner + step;
                if (__shfl_sync(kFull, excl, cand) <= k) owner = cand;
            }
            const int64_t so = __shfl_sync(kFull, s0, owner);
            const int64_t eo = __shfl_sync(kFull, excl, owner);
            if (k < total) {
                const int32_t v = col[so + (k - eo)];
                if (v >= 0 && v < n) {
                    const unsigned long long kv = ((unsigned long long)key[v] << 32) |
                                                  (unsigned long long)(0xffffffffu - (uint32_t)v);
                    atomicMax(&s_best[wbase + owner], kv);
                } else {
                    record_error(st, GB_ERR_RANGE, 12, v);
                }
            }
        }
        __syncwarp();
        const unsigned long long best = s_best[threadIdx.x];
        if (r < n) hub[r] = best ? (int32_t)(0xffffffffu - (uint32_t)(best & 0xffffffffull)) : -1;
        __syncwarp();
    }
}

}  // namespace

namespace {

// ---- The degree-ordered copy of a CSR (for the batched search) -----------
// Its vertex i is original vertex perm[i], in order of decreasing degree (ties
// by id: a stable sort), so the masks of the few vertices that hold most of a
// Kronecker graph's edge endpoints lie together.  Each row keeps its original
// entry order (entries renamed), so the first neighbour of a row in the copy is
// still its smallest original id.
constexpr int RL_THREADS = 512;
constexpr int RL_ITEMS = 16;
constexpr int RL_TILE = RL_THREADS * RL_ITEMS;  // offsets per scan tile
constexpr int64_t RL_LONG = 4096;               // rows copied by a whole block

__global__ void rl_key_kernel(const int64_t *__restrict__ off, int64_t n, uint64_t *__restrict__ key,
                              uint32_t *__restrict__ val)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t d = off[v + 1] - off[v];
        key[v] = 0xffffffffull - (uint64_t)(d < 0xffffffffll ? d : 0xffffffffll);  // ascending = by degree, down
        val[v] = (uint32_t)v;
    }
}

// perm and inv from the sorted ids; dnew[i] = degree of perm[i]
__global__ void rl_perm_kernel(const uint32_t *__restrict__ sorted, const int64_t *__restrict__ off, int64_t n,
                               int32_t *__restrict__ perm, int32_t *__restrict__ inv, int64_t *__restrict__ dnew)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t v = sorted[i];
        perm[i] = (int32_t)v;
        inv[v] = (int32_t)i;
        dnew[i] = off[v + 1] - off[v];
    }
}

// Exclusive scan of dnew into rl_off: tile sums, a scan of the tile sums
// (one block), then each tile scans itself from its base.
__global__ void __launch_bounds__(RL_THREADS) rl_tile_sum_kernel(const int64_t *__restrict__ d, int64_t n,
                                                                 unsigned long long *__restrict__ tsum)
{
    __shared__ unsigned long long s_w[RL_THREADS / 32];
    const int64_t t0 = (int64_t)blockIdx.x * RL_TILE;
    unsigned long long c = 0;
    for (int j = 0; j < RL_ITEMS; ++j) {
        const int64_t i = t0 + (int64_t)j * RL_THREADS + threadIdx.x;
        if (i < n) c += (unsigned long long)d[i];
    }
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < RL_THREADS / 32; ++w) t += s_w[w];
        tsum[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) rl_tile_scan_kernel(const unsigned long long *__restrict__ tsum,
                                                            int64_t ntiles, unsigned long long *__restrict__ tbase)
{
    __shared__ unsigned long long s_w[32];
    const int tid = threadIdx.x;
    const int64_t per = (ntiles + blockDim.x - 1) / blockDim.x;
    const int64_t b0 = (int64_t)tid * per < ntiles ? (int64_t)tid * per : ntiles;
    const int64_t e = b0 + per < ntiles ? b0 + per : ntiles;
    unsigned long long sum = 0;
    for (int64_t i = b0; i < e; ++i) sum += tsum[i];
    const unsigned long long incl = warp_inclusive_scan(sum);
    if ((tid & 31) == 31) s_w[tid >> 5] = incl;
    __syncthreads();
    if (tid < 32) {
        const unsigned long long w = s_w[tid];
        s_w[tid] = warp_inclusive_scan(w) - w;
    }
    __syncthreads();
    unsigned long long run = s_w[tid >> 5] + incl - sum;
    for (int64_t i = b0; i < e; ++i) {
        tbase[i] = run;
        run += tsum[i];
    }
}

__global__ void __launch_bounds__(RL_THREADS) rl_tile_write_kernel(const int64_t *__restrict__ d, int64_t n,
                                                                   const unsigned long long *__restrict__ tbase,
                                                                   int64_t *__restrict__ rl_off)
{
    __shared__ unsigned long long s_w[RL_THREADS / 32];
    // thread t takes RL_ITEMS consecutive entries of the tile
    const int64_t i0 = (int64_t)blockIdx.x * RL_TILE + (int64_t)threadIdx.x * RL_ITEMS;
    unsigned long long own = 0;
    for (int j = 0; j < RL_ITEMS; ++j)
        if (i0 + j < n) own += (unsigned long long)d[i0 + j];
    const unsigned long long incl = warp_inclusive_scan(own);
    if ((threadIdx.x & 31) == 31) s_w[threadIdx.x >> 5] = incl;
    __syncthreads();
    if (threadIdx.x < 32) {
        const unsigned long long w = threadIdx.x < RL_THREADS / 32 ? s_w[threadIdx.x] : 0ull;
        const unsigned long long x = warp_inclusive_scan(w) - w;
        if (threadIdx.x < RL_THREADS / 32) s_w[threadIdx.x] = x;
    }
    __syncthreads();
    unsigned long long run = tbase[blockIdx.x] + s_w[threadIdx.x >> 5] + incl - own;
    for (int j = 0; j < RL_ITEMS; ++j)
        if (i0 + j < n) {
            rl_off[i0 + j] = (int64_t)run;
            run += (unsigned long long)d[i0 + j];
        }
}

// Rows of at most RL_LONG entries: a warp takes 32 rows and streams their
// entries as one sequence (lane k of a round copies entry k), renaming each.
__global__ void rl_copy_rows_kernel(const int64_t *__restrict__ off, const int32_t *__restrict__ col,
                                    const int32_t *__restrict__ perm, const int32_t *__restrict__ inv,
                                    const int64_t *__restrict__ rl_off, int64_t n, int32_t *__restrict__ rl_col)
{
    const unsigned lane = threadIdx.x & 31u;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r0 = gwarp * 32; r0 < n; r0 += nwarps * 32) {
        const int64_t r = r0 + lane;
        int64_t src = 0, dst = 0, d = 0;
        if (r < n) {
            dst = rl_off[r];
            d = rl_off[r + 1] - dst;
            src = off[perm[r]];
            if (d > RL_LONG) d = 0;  // copied by rl_copy_long_kernel
        }
        const int64_t incl = warp_inclusive_scan(d);
        const int64_t total = __shfl_sync(kFull, incl, 31);
        const int64_t excl = incl - d;
        for (int64_t b = 0; b < total; b += 32) {
            const int64_t k = b + lane;
            int owner = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int cand = owner + step;
                if (__shfl_sync(kFull, excl, cand) <= k) owner = cand;
            }
            const int64_t so = __shfl_sync(kFull, src, owner);
            const int64_t doo = __shfl_sync(kFull, dst, owner);
            const int64_t eo = __shfl_sync(kFull, excl, owner);
            if (k < total) rl_col[doo + (k - eo)] = inv[col[so + (k - eo)]];
        }
    }
}

// Rows longer than RL_LONG (the first rows of the copy): one block each.
__global__ void rl_copy_long_kernel(const int64_t *__restrict__ off, const int32_t *__restrict__ col,
                                    const int32_t *__restrict__ perm, const int32_t *__restrict__ inv,
                                    const int64_t *__restrict__ rl_off, int64_t nlong, int32_t *__restrict__ rl_col)
{
    for (int64_t r = blockIdx.x; r < nlong; r += gridDim.x) {
        const int64_t dst = rl_off[r];
        const int64_t d = rl_off[r + 1] - dst;
        if (d <= RL_LONG) continue;
        const int64_t src = off[perm[r]];
        for (int64_t k = threadIdx.x; k < d; k += blockDim.x) rl_col[dst + k] = inv[col[src + k]];
    }
}

}  // namespace

gb_status build_batched_layout(gb_graph *g, cudaStream_t s)
{
    Context *ctx = context();
    if (!ctx) return GB_ERR_CUDA;
    const int64_t n = g->n;
    if (g->rl_col || n == 0) return GB_OK;
    if (n >= (int64_t(1) << 31)) {
        set_error("batched layout: more than 2^31 vertices");
        return GB_ERR_RANGE;
    }
    gb_graph tmpg;  // the new arrays, moved into g once all are built
    Scratch tmp(s);
    uint64_t *k0 = nullptr, *k1 = nullptr;
    uint32_t *v0 = nullptr, *v1 = nullptr;
    GB_CUDA(tmp.alloc(&k0, (size_t)n));
    GB_CUDA(tmp.alloc(&k1, (size_t)n));
    GB_CUDA(tmp.alloc(&v0, (size_t)n));
    GB_CUDA(tmp.alloc(&v1, (size_t)n));
    rl_key_kernel<<<ctx->num_sms * 8, 256, 0, s>>>(g->off, n, k0, v0);
    note_launch();
    GB_CUDA(cudaGetLastError());
    uint64_t *ks = nullptr;
    uint32_t *vs = nullptr;
    gb_status rc = radix_sort(k0, k1, v0, v1, n, 0, 32, &ks, &vs, s);
    if (rc != GB_OK) return rc;
    int64_t *dnew = reinterpret_cast<int64_t *>(ks == k0 ? k1 : k0);  // the sort's spare buffer
    auto fail = [&](cudaError_t e) {
        void *arrays[] = {tmpg.rl_off, tmpg.rl_col, tmpg.rl_perm, tmpg.rl_inv};
        for (void *p : arrays)
            if (p) gb::dfree(p);
        return cuda_fail(e, "batched layout");
    };
    cudaError_t e;
    if ((e = gb::dmalloc(&tmpg.rl_perm, (size_t)n * sizeof(int32_t))) != cudaSuccess ||
        (e = gb::dmalloc(&tmpg.rl_inv, (size_t)n * sizeof(int32_t))) != cudaSuccess ||
        (e = gb::dmalloc(&tmpg.rl_off, (size_t)(n + 1) * sizeof(int64_t))) != cudaSuccess ||
        (e = gb::dmalloc(&tmpg.rl_col, (size_t)col_alloc_entries(g->nnz) * sizeof(int32_t))) != cudaSuccess)
        return fail(e);
    rl_perm_kernel<<<ctx->num_sms * 8, 256, 0, s>>>(vs, g->off, n, tmpg.rl_perm, tmpg.rl_inv, dnew);
    note_launch();
    const int64_t ntiles = (n + RL_TILE - 1) / RL_TILE;
    unsigned long long *tsum = nullptr, *tbase = nullptr;
    if ((e = tmp.alloc(&tsum, (size_t)ntiles)) != cudaSuccess || (e = tmp.alloc(&tbase, (size_t)ntiles)) != cudaSuccess)
        return fail(e);
    rl_tile_sum_kernel<<<(unsigned)ntiles, RL_THREADS, 0, s>>>(dnew, n, tsum);
    note_launch();
    rl_tile_scan_kernel<<<1, 1024, 0, s>>>(tsum, ntiles, tbase);
    note_launch();
    rl_tile_write_kernel<<<(unsigned)ntiles, RL_THREADS, 0, s>>>(dnew, n, tbase, tmpg.rl_off);
    note_launch();
    const int64_t nnz = g->nnz;
    if ((e = cudaMemcpyAsync(tmpg.rl_off + n, &g->nnz, sizeof(int64_t), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail(e);
    (void)nnz;
    rl_copy_rows_kernel<<<ctx->num_sms * 8, 256, 0, s>>>(g->off, g->col, tmpg.rl_perm, tmpg.rl_inv, tmpg.rl_off,
                                                         n, tmpg.rl_col);
    note_launch();
    // the long rows are the first ones of the copy; a block per row up to the
    // first that is not long (each block skips the short ones)
    rl_copy_long_kernel<<<ctx->num_sms * 4, 512, 0, s>>>(g->off, g->col, tmpg.rl_perm, tmpg.rl_inv, tmpg.rl_off,
                                                          std::min<int64_t>(n, g->nnz / (RL_LONG + 1) + 1),
                                                          tmpg.rl_col);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    g->rl_perm = tmpg.rl_perm;
    g->rl_inv = tmpg.rl_inv;
    g->rl_off = tmpg.rl_off;
    g->rl_col = tmpg.rl_col;
    tmpg.rl_perm = tmpg.rl_inv = nullptr;
    tmpg.rl_off = nullptr;
    tmpg.rl_col = nullptr;
    return GB_OK;
}

gb_status build_graph_aux(gb_graph *g, cudaStream_t s)
{
    Context *ctx = context();
    if (!ctx) return GB_ERR_CUDA;
    const int64_t nw = (g->n + 31) / 32;
    GB_CUDA(gb::dmalloc(&g->nz, nw * sizeof(uint32_t)));
    nz_bitmap_kernel<<<ctx->num_sms * 4, 256, 0, s>>>(g->off, g->n, g->nz, nw);
    note_launch();
    GB_CUDA(cudaGetLastError());
    Scratch tmp(s);
    {
        const int64_t nb = (nw + NZL_WORDS - 1) / NZL_WORDS;
        unsigned *cnt = nullptr;
        unsigned long long *base = nullptr;
        GB_CUDA(tmp.alloc(&cnt, (size_t)nb));
        GB_CUDA(tmp.alloc(&base, (size_t)nb + 1));
        nzl_count_kernel<<<(unsigned)nb, NZL_WORDS, 0, s>>>(g->nz, nw, cnt);
        note_launch();
        k1_scan_tiles_kernel<<<1, 1024, 0, s>>>(cnt, nb, base);
        note_launch();
        GB_CUDA(cudaGetLastError());
        unsigned long long nnzv = 0;
        GB_CUDA(cudaMemcpyAsync(&nnzv, base + nb, sizeof(nnzv), cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaStreamSynchronize(s));
        g->nnzv = (int64_t)nnzv;
        GB_CUDA(gb::dmalloc(&g->nzl, std::max<int64_t>(g->nnzv, 4) * sizeof(int32_t)));
        nzl_write_kernel<<<(unsigned)nb, NZL_WORDS, 0, s>>>(g->nz, nw, base, g->nzl);
        note_launch();
        GB_CUDA(cudaGetLastError());
    }
    GB_CUDA(gb::dmalloc(&g->hub, std::max<int64_t>(g->n, 1) * sizeof(int32_t)));
    uint8_t *key = nullptr;
    GB_CUDA(tmp.alloc(&key, (size_t)g->n));
    deg_key_kernel<<<ctx->num_sms * 4, 256, 0, s>>>(g->off, g->n, key);
    note_launch();
    hub_kernel<<<ctx->num_sms * 8, HUB_THREADS, 0, s>>>(g->off, g->col, key, g->n, g->nnz, g->hub,
                                                        ctx->status);
    note_launch();
    GB_CUDA(gb::dmalloc(&g->hd, std::max<int64_t>(g->n, 1) * sizeof(int2)));
    hd_kernel<<<ctx->num_sms * 8, 256, 0, s>>>(g->off, g->hub, g->n, g->hd);
    note_launch();
    GB_CUDA(cudaGetLastError());
    return GB_OK;
}

namespace {

// Stages 2-4 on the symmetrised keys k0[0..nk) (k1: the sort's second buffer
// of nk keys; the caller owns both).
gb_status csr_from_keys(uint64_t *k0, uint64_t *k1, int64_t nk, int scale, gb_graph *g,
                        cudaStream_t s, const unsigned long long *hist = nullptr)
{
    Context *ctx = context();
    const int64_t n = g->n;
    uint64_t *ks = nullptr;
    gb_status rc = radix_sort(k0, k1, nullptr, nullptr, nk, 0, 2 * scale, &ks, nullptr, s, hist);
    if (rc != GB_OK) return rc;
    const int64_t ntiles = (nk + FIN_TILE - 1) / FIN_TILE;
    unsigned *tcnt = nullptr, *wcnt = nullptr;
    unsigned long long *tbase = nullptr;
    Scratch tmp(s);
    GB_CUDA(tmp.alloc(&tcnt, (size_t)ntiles));
    GB_CUDA(tmp.alloc(&wcnt, (size_t)ntiles * FIN_WARPS));
    GB_CUDA(tmp.alloc(&tbase, (size_t)ntiles + 1));
    k1_count_kernel<<<(unsigned)ntiles, FIN_THREADS, 0, s>>>(ks, nk, scale, tcnt, wcnt);
    note_launch();
    k1_scan_tiles_kernel<<<1, 1024, 0, s>>>(tcnt, ntiles, tbase);
    note_launch();
    GB_CUDA(cudaGetLastError());
    unsigned long long nnz = 0;
    DevStatus hst;
    GB_CUDA(cudaMemcpyAsync(&nnz, tbase + ntiles, sizeof(nnz), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaMemcpyAsync(&hst, ctx->status, sizeof(hst), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    if (hst.code != 0) {
        GB_CUDA(cudaMemsetAsync(ctx->status, 0, sizeof(DevStatus), s));
        set_error(hst.code == GB_ERR_RANGE ? "graph_build_csr: an edge endpoint is outside [0, 2^scale)"
                                           : "graph_build_csr: device error during the build");
        return (gb_status)hst.code;
    }
    g->nnz = (int64_t)nnz;
    GB_CUDA(gb::dmalloc(&g->off, (n + 1) * sizeof(int64_t)));
    GB_CUDA(gb::dmalloc(&g->col, col_alloc_entries(g->nnz) * sizeof(int32_t)));
    k1_write_kernel<<<(unsigned)ntiles, FIN_THREADS, 0, s>>>(ks, nk, scale, tbase, wcnt, n, g->off,
                                                             g->col, g->nnz, ctx->status);
    note_launch();
    GB_CUDA(cudaGetLastError());
    return build_graph_aux(g, s);
}

// The graph with no tuples: every row empty.
gb_status empty_csr(gb_graph *g, cudaStream_t s)
{
    g->nnz = 0;
    GB_CUDA(gb::dmalloc(&g->off, (g->n + 1) * sizeof(int64_t)));
    GB_CUDA(gb::dmalloc(&g->col, 16));
    GB_CUDA(cudaMemsetAsync(g->off, 0, (g->n + 1) * sizeof(int64_t), s));
    gb_status r0 = build_graph_aux(g, s);
    if (r0 != GB_OK) return r0;
    GB_CUDA(cudaStreamSynchronize(s));
    return GB_OK;
}

}  // namespace

gb_status build_csr(const int64_t *edges, int64_t m, int scale, gb_graph *g, cudaStream_t s)
{
    Context *ctx = context();
    if (!ctx) return GB_ERR_CUDA;
    const int64_t nk = 2 * m;
    g->n = int64_t(1) << scale;
    g->scale = scale;
    g->device = ctx->device;
    GB_CUDA(cudaMemsetAsync(ctx->status, 0, sizeof(DevStatus), s));
    if (nk == 0) return empty_csr(g, s);
    uint64_t *k0 = nullptr, *k1 = nullptr;
    unsigned long long *hist = nullptr;
    SortPlan plan = sort_plan(0, 2 * scale);
    Scratch tmp(s);
    GB_CUDA(tmp.alloc(&k0, (size_t)nk));
    GB_CUDA(tmp.alloc(&k1, (size_t)nk));
    if (plan.passes > RS_MAX_PASSES) {
        plan.passes = 0;  // the sort counts (and rejects) it
    } else {
        GB_CUDA(tmp.alloc(&hist, (size_t)plan.passes * RS_RADIX_MAX));
        GB_CUDA(cudaMemsetAsync(hist, 0, (size_t)plan.passes * RS_RADIX_MAX * sizeof(unsigned long long), s));
    }
    k1_sym_kernel<<<ctx->num_sms * 8, SYM_THREADS, 0, s>>>(edges, m, scale, reinterpret_cast<ulonglong2 *>(k0),
                                                           plan, hist, ctx->status);
    note_launch();
    GB_CUDA(cudaGetLastError());
    return csr_from_keys(k0, k1, nk, scale, g, s, hist);
}

gb_status kron_csr(int scale, int edgefactor, double a, double b, double c, uint64_t seed_gen,
                   uint64_t seed_perm, gb_graph *g, cudaStream_t s)
{
    Context *ctx = context();
    if (!ctx) return GB_ERR_CUDA;
    if (scale < 1 || scale > 30 || edgefactor < 1) {
        set_error("graph_generate_csr: need 1 <= scale <= 30, edgefactor >= 1");
        return GB_ERR_INVALID;
    }
    if ((int64_t(1) << scale) * edgefactor > (int64_t(1) << 32)) {
        set_error("graph_generate_csr: more than 2^32 tuples");
        return GB_ERR_RANGE;
    }
    const int64_t nk = 2 * ((int64_t(1) << scale) * edgefactor);
    g->n = int64_t(1) << scale;
    g->scale = scale;
    g->device = ctx->device;
    GB_CUDA(cudaMemsetAsync(ctx->status, 0, sizeof(DevStatus), s));
    uint64_t *k0 = nullptr, *k1 = nullptr;
    Scratch tmp(s);
    GB_CUDA(tmp.alloc(&k0, (size_t)nk));
    GB_CUDA(tmp.alloc(&k1, (size_t)nk));
    gb_status rc = kron_keys_impl(scale, edgefactor, a, b, c, seed_gen, seed_perm, k0, s);
    if (rc != GB_OK) return rc;
    return csr_from_keys(k0, k1, nk, scale, g, s);
}

// ---------------------------------------------------------------------------
// Kernel 1, counting-sort variant (a comparison path for the radix build):
//   1. entries per row, self-loops skipped and duplicates counted (atomics);
//   2. an exclusive scan gives each row its start s0 in a scratch column array;
//   3. every tuple's two endpoints are scattered into their rows;
//   4. every row is sorted in place and its distinct entries counted: rows of
//      at most 32 entries by one warp (a bitonic network over shuffles), rows of
//      at most CS_BLOCK_MAX by one block (a bitonic network in shared memory),
//      longer rows by one device radix sort of (row rank, column) keys;
//   5. a scan of the distinct counts gives the offsets, and one warp per row
//      copies the row's distinct entries to the columns.
// The result is the same CSR as the radix build, bit for bit.
// ---------------------------------------------------------------------------
namespace {

constexpr int CS_THREADS = 256;
constexpr int CS_CHUNK = CS_THREADS * 16;   // elements per block of the scans
constexpr int CS_BLOCK_MAX = 4096;          // longest row sorted in shared memory
constexpr int SITE_CS = 14;

__global__ void cs_count_kernel(const int64_t *__restrict__ edges, int64_t m, int64_t n,
                                unsigned *__restrict__ deg0, DevStatus *st)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int64_t u = edges[e], v = edges[m + e];
        if (u < 0 || u >= n || v < 0 || v >= n) {
            record_error(st, GB_ERR_RANGE, SITE_K1_RANGE, (long long)e);
            continue;
        }
        if (u == v) continue;
        atomicAdd(&deg0[u], 1u);
        atomicAdd(&deg0[v], 1u);
    }
}

// Exclusive scan of cnt[0..n) into out[0..n] (out[n] = total), three steps:
// chunk sums, a scan of the chunk sums, the chunks rescanned from their bases.
__global__ void __launch_bounds__(CS_THREADS) cs_chunk_sum_kernel(const unsigned *__restrict__ cnt,
                                                                  int64_t n, unsigned *__restrict__ sums)
{
    __shared__ unsigned long long s_w[CS_THREADS / 32];
    const int64_t c0 = (int64_t)blockIdx.x * CS_CHUNK;
    unsigned long long t = 0;
    for (int j = 0; j < CS_CHUNK / CS_THREADS; ++j) {
        const int64_t i = c0 + (int64_t)j * CS_THREADS + threadIdx.x;
        if (i < n) t += cnt[i];
    }
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = 0;
        for (int w = 0; w < CS_THREADS / 32; ++w) b += s_w[w];
        sums[blockIdx.x] = (unsigned)b;  // at most 2m < 2^32 entries in all
    }
}

__global__ void __launch_bounds__(CS_THREADS) cs_chunk_write_kernel(
    const unsigned *__restrict__ cnt, int64_t n, const unsigned long long *__restrict__ base,
    int64_t nchunks, int64_t *__restrict__ out)
{
    __shared__ unsigned long long s_w[CS_THREADS / 32];
    constexpr int PER = CS_CHUNK / CS_THREADS;  // 16 consecutive elements per thread
    const int64_t i0 = (int64_t)blockIdx.x * CS_CHUNK + (int64_t)threadIdx.x * PER;
    unsigned long long t = 0;
    for (int j = 0; j < PER; ++j)
        if (i0 + j < n) t += cnt[i0 + j];
    const unsigned long long incl = warp_inclusive_scan(t);
    if ((threadIdx.x & 31) == 31) s_w[threadIdx.x >> 5] = incl;
    __syncthreads();
    unsigned long long run = base[blockIdx.x] + incl - t;
    for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) run += s_w[w];
    for (int j = 0; j < PER; ++j) {
        if (i0 + j < n) {
            out[i0 + j] = (int64_t)run;
            run += cnt[i0 + j];
        }
    }
    if (blockIdx.x == nchunks - 1 && threadIdx.x == 0) out[n] = (int64_t)base[nchunks];
}

__global__ void cs_scatter_kernel(const int64_t *__restrict__ edges, int64_t m, int64_t n,
                                  const int64_t *__restrict__ s0, unsigned *__restrict__ fill,
                                  int32_t *__restrict__ tmp, DevStatus *st)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int64_t u = edges[e], v = edges[m + e];
        if (u < 0 || u >= n || v < 0 || v >= n || u == v) continue;
        const int64_t p = s0[u] + atomicAdd(&fill[u], 1u);
        const int64_t q = s0[v] + atomicAdd(&fill[v], 1u);
        if (p < s0[u + 1]) tmp[p] = (int32_t)v;
        else record_error(st, GB_ERR_RANGE, SITE_CS, p);
        if (q < s0[v + 1]) tmp[q] = (int32_t)u;
        else record_error(st, GB_ERR_RANGE, SITE_CS, q);
    }
}

// Rows by length: <= 1 (already sorted: its distinct count is its length),
// <= 32, <= CS_BLOCK_MAX, longer; the last three appended to their lists.
__global__ void cs_classify_kernel(const int64_t *__restrict__ s0, int64_t n,
                                   unsigned *__restrict__ dcnt, int32_t *__restrict__ lists,
                                   unsigned long long *__restrict__ counts)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x0 = (int64_t)blockIdx.x * blockDim.x; x0 < n; x0 += stride) {
        const int64_t x = x0 + threadIdx.x;
        const int64_t len = x < n ? s0[x + 1] - s0[x] : 0;
        int cls = -1;
        if (x < n) {
            if (len <= 1) dcnt[x] = (unsigned)len;
            else cls = len <= 32 ? 0 : (len <= CS_BLOCK_MAX ? 1 : 2);
        }
        for (int c = 0; c < 3; ++c) {
            const unsigned bm = __ballot_sync(kFull, cls == c);
            if (!bm) continue;
            unsigned long long b = 0;
            if ((threadIdx.x & 31) == 0) b = atomicAdd(&counts[c], (unsigned long long)__popc(bm));
            b = __shfl_sync(kFull, b, 0);
            if (cls == c) lists[(int64_t)c * n + (int64_t)b + __popc(bm & lanemask_lt())] = (int32_t)x;
        }
    }
}

// Rows of 2..32 entries: one warp per row, a bitonic network over shuffles.
__global__ void cs_sort_warp_kernel(const int32_t *__restrict__ rows, int64_t nrows,
                                    const int64_t *__restrict__ s0, int32_t *__restrict__ tmp,
                                    unsigned *__restrict__ dcnt)
{
    const unsigned lane = threadIdx.x & 31u;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = gwarp; r < nrows; r += nwarps) {
        const int32_t x = rows[r];
        const int64_t s = s0[x];
        const int len = (int)(s0[x + 1] - s);
        int32_t val = (int)lane < len ? tmp[s + lane] : 0x7fffffff;
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const int32_t other = __shfl_xor_sync(kFull, val, j);
                const bool up = (lane & k) == 0, lower = (lane & j) == 0;
                val = (lower == up) ? min(val, other) : max(val, other);
            }
        }
        const int32_t prev = __shfl_up_sync(kFull, val, 1);
        const unsigned firsts = __ballot_sync(kFull, (int)lane < len && (lane == 0 || prev != val));
        if ((int)lane < len) tmp[s + lane] = val;
        if (lane == 0) dcnt[x] = __popc(firsts);
    }
}

// Rows of 33..CS_BLOCK_MAX entries: one block per row, a bitonic network in
// shared memory over the next power of two (padded with the largest int).
__global__ void __launch_bounds__(CS_THREADS) cs_sort_block_kernel(
    const int32_t *__restrict__ rows, int64_t nrows, const int64_t *__restrict__ s0,
    int32_t *__restrict__ tmp, unsigned *__restrict__ dcnt)
{
    __shared__ int32_t buf[CS_BLOCK_MAX];
    __shared__ unsigned s_w[CS_THREADS / 32];
    for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int32_t x = rows[r];
        const int64_t s = s0[x];
        const int len = (int)(s0[x + 1] - s);
        int p2 = 64;
        while (p2 < len) p2 <<= 1;
        for (int i = threadIdx.x; i < p2; i += CS_THREADS) buf[i] = i < len ? tmp[s + i] : 0x7fffffff;
        __syncthreads();
        for (int k = 2; k <= p2; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < p2; i += CS_THREADS) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const int32_t a = buf[i], b = buf[ixj];
                        if ((a > b) == ((i & k) == 0)) {
                            buf[i] = b;
                            buf[ixj] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        unsigned c = 0;
        for (int i = threadIdx.x; i < len; i += CS_THREADS) {
            tmp[s + i] = buf[i];
            c += (i == 0 || buf[i] != buf[i - 1]);
        }
        c = warp_sum(c);
        if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned t = 0;
            for (int w = 0; w < CS_THREADS / 32; ++w) t += s_w[w];
            dcnt[x] = t;
        }
        __syncthreads();  // buf and s_w are reused by the next row
    }
}

// Long rows: the lengths of the listed rows (for their scan).
__global__ void cs_long_len_kernel(const int32_t *__restrict__ rows, int64_t nrows,
                                   const int64_t *__restrict__ s0, unsigned *__restrict__ len)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += stride) {
        const int32_t x = rows[r];
        len[r] = (unsigned)(s0[x + 1] - s0[x]);
    }
}

// Long rows, before and after their sort: keys (rank << scale | column) are
// gathered at the row's place g0[rank], and written back in sorted order with
// the distinct count.  One block per row.
__global__ void __launch_bounds__(CS_THREADS) cs_long_gather_kernel(
    const int32_t *__restrict__ rows, int64_t nrows, const int64_t *__restrict__ s0,
    const int64_t *__restrict__ g0, const int32_t *__restrict__ tmp, int scale,
    uint64_t *__restrict__ keys)
{
    for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int32_t x = rows[r];
        const int64_t s = s0[x], len = s0[x + 1] - s, g = g0[r];
        for (int64_t i = threadIdx.x; i < len; i += CS_THREADS)
            keys[g + i] = ((uint64_t)r << scale) | (uint64_t)(uint32_t)tmp[s + i];
    }
}

__global__ void __launch_bounds__(CS_THREADS) cs_long_scatter_kernel(
    const int32_t *__restrict__ rows, int64_t nrows, const int64_t *__restrict__ s0,
    const int64_t *__restrict__ g0, const uint64_t *__restrict__ keys, int scale,
    int32_t *__restrict__ tmp, unsigned *__restrict__ dcnt)
{
    __shared__ unsigned s_w[CS_THREADS / 32];
    const uint64_t vmask = (uint64_t(1) << scale) - 1;
    for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int32_t x = rows[r];
        const int64_t s = s0[x], len = s0[x + 1] - s, g = g0[r];
        unsigned c = 0;
        for (int64_t i = threadIdx.x; i < len; i += CS_THREADS) {
            const uint64_t k = keys[g + i];
            tmp[s + i] = (int32_t)(k & vmask);
            c += (i == 0 || keys[g + i - 1] != k);
        }
        c = warp_sum(c);
        if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned t = 0;
            for (int w = 0; w < CS_THREADS / 32; ++w) t += s_w[w];
            dcnt[x] = t;
        }
        __syncthreads();
    }
}

// Each row's distinct entries (its sorted scratch run without repeats) to the
// columns at off[x]; one warp per row.
__global__ void cs_compact_kernel(const int64_t *__restrict__ s0, const int64_t *__restrict__ off,
                                  int64_t n, const int32_t *__restrict__ tmp,
                                  int32_t *__restrict__ col, int64_t nnz, DevStatus *st)
{
    const unsigned lane = threadIdx.x & 31u;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = gwarp; x < n; x += nwarps) {
        const int64_t s = s0[x], len = s0[x + 1] - s;
        int64_t pos = off[x];
        int32_t last = -1;  // the row's previous entry (columns are >= 0)
        for (int64_t i0 = 0; i0 < len; i0 += 32) {
            const int64_t i = i0 + lane;
            const int32_t v = i < len ? tmp[s + i] : -1;
            int32_t pv = __shfl_up_sync(kFull, v, 1);
            if (lane == 0) pv = last;
            const bool first = i < len && v != pv;
            const unsigned fm = __ballot_sync(kFull, first);
            if (first) {
                const int64_t p = pos + __popc(fm & lanemask_lt());
                if (p < nnz) col[p] = v;
                else record_error(st, GB_ERR_RANGE, SITE_CS, p);
            }
            pos += __popc(fm);
            last = __shfl_sync(kFull, v, 31);
        }
    }
}

// out[0..n] = exclusive scan of cnt[0..n); synchronises nothing.
gb_status cs_scan(const unsigned *cnt, int64_t n, int64_t *out, cudaStream_t s)
{
    const int64_t nchunks = std::max<int64_t>(1, (n + CS_CHUNK - 1) / CS_CHUNK);
    unsigned *sums = nullptr;
    unsigned long long *base = nullptr;
    Scratch tmp(s);
    GB_CUDA(tmp.alloc(&sums, (size_t)nchunks));
    GB_CUDA(tmp.alloc(&base, (size_t)nchunks + 1));
    cs_chunk_sum_kernel<<<(unsigned)nchunks, CS_THREADS, 0, s>>>(cnt, n, sums);
    note_launch();
    k1_scan_tiles_kernel<<<1, 1024, 0, s>>>(sums, nchunks, base);
    note_launch();
    cs_chunk_write_kernel<<<(unsigned)nchunks, CS_THREADS, 0, s>>>(cnt, n, base, nchunks, out);
    note_launch();
    GB_CUDA(cudaGetLastError());
    return GB_OK;
}

}  // namespace

gb_status build_csr_counting(const int64_t *edges, int64_t m, int scale, gb_graph *g,
                             cudaStream_t s)
{
    Context *ctx = context();
    if (!ctx) return GB_ERR_CUDA;
    const int64_t n = int64_t(1) << scale;
    g->n = n;
    g->scale = scale;
    g->device = ctx->device;
    if (m >= (int64_t(1) << 31)) {  // 32-bit row counts hold at most 2m < 2^32 entries
        set_error("graph_build_csr_counting: needs m < 2^31 tuples");
        return GB_ERR_RANGE;
    }
    GB_CUDA(cudaMemsetAsync(ctx->status, 0, sizeof(DevStatus), s));
    if (m == 0) return empty_csr(g, s);
    const int grid = ctx->num_sms * 8;
    unsigned *cnt = nullptr, *dcnt = nullptr;
    int64_t *s0 = nullptr;
    Scratch scr(s);
    GB_CUDA(scr.alloc(&cnt, (size_t)n));
    GB_CUDA(scr.alloc(&dcnt, (size_t)n));
    GB_CUDA(scr.alloc(&s0, (size_t)n + 1));
    // 1-2: entries per row, then the row starts
    GB_CUDA(cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(unsigned), s));
    cs_count_kernel<<<grid, 256, 0, s>>>(edges, m, n, cnt, ctx->status);
    note_launch();
    gb_status rc = cs_scan(cnt, n, s0, s);
    if (rc != GB_OK) return rc;
    int64_t nnz0 = 0;
    DevStatus hst;
    GB_CUDA(cudaMemcpyAsync(&nnz0, s0 + n, sizeof(nnz0), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaMemcpyAsync(&hst, ctx->status, sizeof(hst), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    if (hst.code != 0) {
        GB_CUDA(cudaMemsetAsync(ctx->status, 0, sizeof(DevStatus), s));
        set_error(hst.code == GB_ERR_RANGE ? "graph_build_csr_counting: an edge endpoint is outside [0, 2^scale)"
                                           : "graph_build_csr_counting: device error during the build");
        return (gb_status)hst.code;
    }
    // 3: scatter into the rows (cnt reused as the fill counters)
    int32_t *tmp = nullptr;
    GB_CUDA(scr.alloc(&tmp, (size_t)std::max<int64_t>(nnz0, 1)));
    GB_CUDA(cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(unsigned), s));
    cs_scatter_kernel<<<grid, 256, 0, s>>>(edges, m, n, s0, cnt, tmp, ctx->status);
    note_launch();
    // 4: rows sorted by length class
    int32_t *lists = nullptr;
    unsigned long long *counts = nullptr;
    GB_CUDA(scr.alloc(&lists, 3 * (size_t)n));
    GB_CUDA(scr.alloc(&counts, 3));
    GB_CUDA(cudaMemsetAsync(counts, 0, 3 * sizeof(unsigned long long), s));
    cs_classify_kernel<<<grid, 256, 0, s>>>(s0, n, dcnt, lists, counts);
    note_launch();
    unsigned long long hc[3];
    GB_CUDA(cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    if (hc[0]) {
        cs_sort_warp_kernel<<<grid, 256, 0, s>>>(lists, (int64_t)hc[0], s0, tmp, dcnt);
        note_launch();
    }
    if (hc[1]) {
        cs_sort_block_kernel<<<(unsigned)std::min<unsigned long long>(hc[1], (unsigned long long)ctx->num_sms * 8),
                               CS_THREADS, 0, s>>>(lists + n, (int64_t)hc[1], s0, tmp, dcnt);
        note_launch();
    }
    if (hc[2]) {
        const int64_t nl = (int64_t)hc[2];
        const int32_t *lrows = lists + 2 * n;
        unsigned *llen = nullptr;
        int64_t *g0 = nullptr;
        Scratch lt(s);  // the long rows' temporaries, freed at the end of this block
        GB_CUDA(lt.alloc(&llen, (size_t)nl));
        GB_CUDA(lt.alloc(&g0, (size_t)nl + 1));
        cs_long_len_kernel<<<grid, 256, 0, s>>>(lrows, nl, s0, llen);
        note_launch();
        rc = cs_scan(llen, nl, g0, s);
        if (rc != GB_OK) return rc;
        int64_t tl = 0;
        GB_CUDA(cudaMemcpyAsync(&tl, g0 + nl, sizeof(tl), cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaStreamSynchronize(s));
        int rbits = 1;
        while ((int64_t(1) << rbits) < nl) ++rbits;
        uint64_t *k0 = nullptr, *k1 = nullptr, *ks = nullptr;
        GB_CUDA(lt.alloc(&k0, (size_t)tl));
        GB_CUDA(lt.alloc(&k1, (size_t)tl));
        const unsigned lb = (unsigned)std::min<int64_t>(nl, (int64_t)ctx->num_sms * 8);
        cs_long_gather_kernel<<<lb, CS_THREADS, 0, s>>>(lrows, nl, s0, g0, tmp, scale, k0);
        note_launch();
        rc = radix_sort(k0, k1, nullptr, nullptr, tl, 0, scale + rbits, &ks, nullptr, s);
        if (rc != GB_OK) return rc;
        cs_long_scatter_kernel<<<lb, CS_THREADS, 0, s>>>(lrows, nl, s0, g0, ks, scale, tmp, dcnt);
        note_launch();
        GB_CUDA(cudaGetLastError());
    }
    // 5: offsets from the distinct counts, then the columns
    GB_CUDA(gb::dmalloc(&g->off, (n + 1) * sizeof(int64_t)));
    rc = cs_scan(dcnt, n, g->off, s);
    if (rc != GB_OK) return rc;
    int64_t nnz = 0;
    GB_CUDA(cudaMemcpyAsync(&nnz, g->off + n, sizeof(nnz), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    g->nnz = nnz;
    GB_CUDA(gb::dmalloc(&g->col, col_alloc_entries(nnz) * sizeof(int32_t)));
    cs_compact_kernel<<<grid, 256, 0, s>>>(s0, g->off, n, tmp, g->col, nnz, ctx->status);
    note_launch();
    GB_CUDA(cudaGetLastError());
    return build_graph_aux(g, s);
}

}  // namespace gb
