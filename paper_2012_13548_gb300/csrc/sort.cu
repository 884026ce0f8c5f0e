// LSD radix sort of uint64 keys (optionally carrying uint32 values) for the
// Kronecker generator (vertex permutation, edge shuffle) and for kernel 1
// (Sec. 2.2 builds the CSR from the edges in sorted order; Sec. 4.2 names a
// parallel sort as the way to build it).
//
// Design (one-sweep, after Adinets & Merrill 2022): one read of the keys
// counts the digits of every pass; then each pass is a single kernel in
// which every tile ranks its keys with warp match-any, publishes its digit
// counts, looks back over earlier tiles (decoupled look-back) for its global
// offsets and scatters through shared memory so that each digit run is
// written contiguously.  Digits are 8 bits wide, or 9 where that saves a
// pass (52 key bits: 4 x 9 + 2 x 8 instead of 7 x 8).  Tiles take their index from an atomic counter, so a
// tile only ever waits on tiles that are already running; every wait is
// bounded and records GB_ERR_TIMEOUT instead of hanging.  Inputs larger than
// one portion (2^28 keys by default, smaller on request) are sorted portion by
// portion, chained through their digit bases, which keeps the look-back values
// within 30 bits.
#include "common.cuh"
#include "internal.h"

#include <algorithm>
#include <atomic>

namespace gb {
namespace {

constexpr int RS_THREADS = 512;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // keys per tile
#define RS_MINB(vals) ((vals) ? 3 * 256 / RS_THREADS : 4 * 256 / RS_THREADS)
static_assert(RS_THREADS % 256 == 0, "threads 0..255 own one digit each");
constexpr int64_t RS_PORTION = int64_t(1) << 28;  // default and largest portion
constexpr unsigned FLAG_AGG = 1u << 30;
constexpr unsigned FLAG_INCL = 2u << 30;
constexpr unsigned VAL_MASK = FLAG_AGG - 1u;
constexpr int RS_R = RS_RADIX_MAX;  // stride of the per-pass digit tables

__global__ void __launch_bounds__(512) rs_hist_kernel(const uint64_t *__restrict__ keys, int64_t n,
                                                      SortPlan plan,
                                                      unsigned long long *__restrict__ hist)
{
    __shared__ unsigned s_h[RS_MAX_PASSES][RS_R];
    for (int i = threadIdx.x; i < RS_MAX_PASSES * RS_R; i += blockDim.x) (&s_h[0][0])[i] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t k = keys[i];
#pragma unroll
        for (int p = 0; p < RS_MAX_PASSES; ++p) {  // unrolled: the plan stays in registers
            if (p >= plan.passes) break;
            atomicAdd(&s_h[p][(unsigned)(k >> plan.shift[p]) & ((1u << plan.bits[p]) - 1u)], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < plan.passes * RS_R; i += blockDim.x) {
        unsigned c = (&s_h[0][0])[i];
        if (c) atomicAdd(&hist[i], (unsigned long long)c);
    }
}

// Exclusive scan of each pass's digit counts into the first portion's bases.
__global__ void __launch_bounds__(RS_R) rs_scan_kernel(const unsigned long long *__restrict__ hist, int passes,
                                                      int64_t portions, unsigned long long *__restrict__ base)
{
    __shared__ unsigned long long s[RS_R];
    const int d = threadIdx.x;
    for (int p = 0; p < passes; ++p) {
        s[d] = hist[p * RS_R + d];
        __syncthreads();
        for (int o = 1; o < RS_R; o <<= 1) {
            unsigned long long t = d >= o ? s[d - o] : 0;
            __syncthreads();
            s[d] += t;
            __syncthreads();
        }
        base[(size_t)p * (portions + 1) * RS_R + d] = s[d] - hist[p * RS_R + d];
        __syncthreads();
    }
}

// Register budget: keys-only passes (kernel 1) keep 1024 threads per SM
// resident, passes that carry values 768 (rounded down to whole blocks); both
// are latency-bound, so resident warps matter.
template <bool VALS, int DBITS>
__global__ void __launch_bounds__(RS_THREADS, RS_MINB(VALS)) rs_onesweep_kernel(
    const uint64_t *__restrict__ kin, uint64_t *__restrict__ kout, const uint32_t *__restrict__ vin,
    uint32_t *__restrict__ vout, int64_t begin, int64_t count, int shift, int ntiles,
    const unsigned long long *__restrict__ base_in, unsigned long long *__restrict__ base_out,
    unsigned *status, DevStatus *st, uint64_t timeout_ns, int64_t n_all)
{
    constexpr int RADIX = 1 << DBITS;
    constexpr unsigned DMASK = RADIX - 1;
    static_assert(RADIX <= RS_THREADS, "one owner thread per digit");
    extern __shared__ __align__(16) unsigned char rs_dyn[];
    uint64_t *s_keys = reinterpret_cast<uint64_t *>(rs_dyn);
    uint32_t *s_vals = reinterpret_cast<uint32_t *>(rs_dyn + RS_TILE * sizeof(uint64_t));
    __shared__ unsigned short s_whist[RS_WARPS][RADIX];
    __shared__ unsigned s_excl[RADIX];
    __shared__ long long s_adj[RADIX];
    __shared__ unsigned s_wsum[RS_WARPS];
    __shared__ unsigned s_tile;
    __shared__ int s_bad;

    const int tid = threadIdx.x;
    const unsigned lane = tid & 31u;
    const int warp = tid >> 5;
    if (tid == 0) {
        s_tile = atomicAdd(&status[0], 1u);
        s_bad = 0;
    }
    for (int i = tid; i < RS_WARPS * RADIX; i += RS_THREADS) (&s_whist[0][0])[i] = 0;
    __syncthreads();
    const int tile = (int)s_tile;
    const int64_t tbase = begin + (int64_t)tile * RS_TILE;
    const int64_t tend = min(begin + count, tbase + (int64_t)RS_TILE);
    const int tn = (int)(tend - tbase);

    // Load warp-striped: item j of this lane is tbase + warp*512 + j*32 + lane.
    uint64_t k[RS_ITEMS];
    uint32_t v[RS_ITEMS];
    unsigned short rk[RS_ITEMS];
    const int64_t wbase = tbase + (int64_t)warp * (32 * RS_ITEMS);
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
        const int64_t idx = wbase + j * 32 + lane;
        k[j] = idx < tend ? kin[idx] : 0ull;
        if (VALS) v[j] = idx < tend ? vin[idx] : 0u;
    }
    // Warp-level stable ranking by digit (multisplit: the lanes holding the same
    // digit found with one ballot per digit bit, faster here than match-any).
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
        const bool valid = wbase + j * 32 + lane < tend;
        const unsigned dg = valid ? (unsigned)(k[j] >> shift) & DMASK : (unsigned)RADIX;
        // lanes with the same digit: one ballot per digit bit (and the valid bit)
        unsigned peers = kFull;
#pragma unroll
        for (int bit = 0; bit <= DBITS; ++bit) {
            const unsigned bl = __ballot_sync(kFull, (dg >> bit) & 1u);
            peers &= ((dg >> bit) & 1u) ? bl : ~bl;
        }
        const unsigned before = __popc(peers & lanemask_lt());
        unsigned cnt = 0;
        if (valid) cnt = s_whist[warp][dg];
        __syncwarp();
        if (valid && before == 0) s_whist[warp][dg] = (unsigned short)(cnt + __popc(peers));
        __syncwarp();
        rk[j] = (unsigned short)(cnt + before);
    }
    __syncthreads();

    // Thread d < RADIX owns digit d: per-warp exclusive offsets and the tile total.
    const int d = tid;
    const bool owner = tid < RADIX;
    unsigned total = 0, incl = 0;
    volatile unsigned *my_status = status + 1 + (size_t)tile * RADIX + (owner ? d : 0);
    if (owner) {
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            const unsigned c = s_whist[w][d];
            s_whist[w][d] = (unsigned short)total;
            total += c;
        }
        *my_status = (tile == 0 ? FLAG_INCL : FLAG_AGG) | total;
        // exclusive scan of the tile totals over digits (warps 0..RADIX/32-1)
        incl = warp_inclusive_scan(total);
        if (lane == 31) s_wsum[warp] = incl;
    }
    __syncthreads();
    if (owner) {
        unsigned woff = 0;
        for (int w = 0; w < warp; ++w) woff += s_wsum[w];
        s_excl[d] = woff + incl - total;

        // Decoupled look-back over earlier tiles for this digit.
        unsigned long long prefix = 0;
        if (tile > 0) {
            int t = tile - 1;
            unsigned spins = 0;
            uint64_t t0 = 0;
            while (true) {
                const unsigned sv = *(volatile const unsigned *)(status + 1 + (size_t)t * RADIX + d);
                if ((sv & ~VAL_MASK) == 0) {
                    if (((++spins) & 63u) == 0) {
                        const uint64_t now = globaltimer_ns();
                        if (t0 == 0) t0 = now;
                        else if (now - t0 > timeout_ns) {
                            record_error(st, GB_ERR_TIMEOUT, 100, (long long)tile);
                            s_bad = 1;
                            break;
                        }
                    }
                    continue;
                }
                prefix += sv & VAL_MASK;
                if (sv & FLAG_INCL) break;
                --t;
                if (t < 0) break;  // tile 0 always publishes FLAG_INCL
            }
            *my_status = FLAG_INCL | (unsigned)((prefix + total) & VAL_MASK);
        }
        const unsigned long long gstart = base_in[d] + prefix;
        if (tile == ntiles - 1) base_out[d] = gstart + total;
        s_adj[d] = (long long)gstart - (long long)s_excl[d];
    }
    __syncthreads();

    // Scatter into shared memory in digit order, then write each run out.
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
        if (wbase + j * 32 + lane < tend) {
            const unsigned dg = (unsigned)(k[j] >> shift) & DMASK;
            const unsigned pos = s_excl[dg] + s_whist[warp][dg] + rk[j];
            s_keys[pos] = k[j];
            if (VALS) s_vals[pos] = v[j];
        }
    }
    __syncthreads();
    if (s_bad) return;  // offsets unknown after a timed-out look-back: write nothing
    for (int i = tid; i < tn; i += RS_THREADS) {
        const uint64_t kk = s_keys[i];
        const long long o = s_adj[(unsigned)(kk >> shift) & DMASK] + i;
        if (o < 0 || o >= n_all) {
            record_error(st, GB_ERR_RANGE, 101, o);
            continue;
        }
        kout[o] = kk;
        if (VALS) vout[o] = s_vals[i];
    }
}

// The shared-memory limits of the sort kernels are raised once per device
// (cudaFuncSetAttribute applies to the device current at the call).
constexpr int kAttrDevices = 64;
std::atomic<bool> g_attr_set[kAttrDevices];

// Keys per portion (gb_set_sort_portion); every portion size gives the same result.
std::atomic<int64_t> g_portion{RS_PORTION};

}  // namespace

gb_status set_sort_portion(int64_t keys)
{
    if (keys < 0 || keys > RS_PORTION) {
        set_error("gb_set_sort_portion: keys must be 0 (the default) or in [1, 2^28]");
        return GB_ERR_INVALID;
    }
    g_portion.store(keys == 0 ? RS_PORTION : keys);
    return GB_OK;
}

int64_t sort_portion() { return g_portion.load(); }

SortPlan sort_plan(int begin_bit, int end_bit)
{
    SortPlan p{};
    const int b = end_bit - begin_bit;
    p.passes = b <= 0 ? 0 : (b + RS_MAX_BITS - 1) / RS_MAX_BITS;
    const int wide = std::max(0, b - 8 * p.passes);  // passes of 9 bits (the others 8)
    int sh = begin_bit;
    for (int i = 0; i < p.passes; ++i) {
        p.bits[i] = i < wide ? 9 : 8;
        p.shift[i] = sh;
        sh += p.bits[i];
    }
    return p;
}

gb_status radix_sort(uint64_t *keys, uint64_t *keys_alt, uint32_t *vals, uint32_t *vals_alt,
                     int64_t n, int begin_bit, int end_bit, uint64_t **keys_out,
                     uint32_t **vals_out, cudaStream_t s, const unsigned long long *hist_in)
{
    *keys_out = keys;
    if (vals_out) *vals_out = vals;
    if (n <= 1 || end_bit <= begin_bit) return GB_OK;
    if (begin_bit < 0 || end_bit > 64) {
        set_error("radix_sort: bad bit range");
        return GB_ERR_INVALID;
    }
    Context *ctx = context();
    if (!ctx) return GB_ERR_CUDA;
    const bool has_vals = vals != nullptr;
    const SortPlan plan = sort_plan(begin_bit, end_bit);
    const int passes = plan.passes;
    const int64_t portion = g_portion.load();
    const int64_t portions = (n + portion - 1) / portion;
    const int64_t tiles_max = (std::min(n, portion) + RS_TILE - 1) / RS_TILE;
    const size_t dyn_smem = RS_TILE * sizeof(uint64_t) + (has_vals ? RS_TILE * sizeof(uint32_t) : 0);
    const bool attr_known = ctx->device >= 0 && ctx->device < kAttrDevices;
    if (!attr_known || !g_attr_set[ctx->device].load()) {
        const int with_vals = (int)(RS_TILE * (sizeof(uint64_t) + sizeof(uint32_t)));
        const int keys_only = (int)(RS_TILE * sizeof(uint64_t));
        GB_CUDA(cudaFuncSetAttribute(rs_onesweep_kernel<true, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     with_vals));
        GB_CUDA(cudaFuncSetAttribute(rs_onesweep_kernel<true, 9>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     with_vals));
        GB_CUDA(cudaFuncSetAttribute(rs_onesweep_kernel<false, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     keys_only));
        GB_CUDA(cudaFuncSetAttribute(rs_onesweep_kernel<false, 9>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     keys_only));
        if (attr_known) g_attr_set[ctx->device].store(true);
    }

    unsigned long long *hist = nullptr, *base = nullptr;
    unsigned *status = nullptr;
    Scratch tmp(s);
    GB_CUDA(tmp.alloc(&base, (size_t)passes * (portions + 1) * RS_R));
    GB_CUDA(tmp.alloc(&status, 1 + (size_t)tiles_max * RS_R));
    if (!hist_in) {
        GB_CUDA(tmp.alloc(&hist, (size_t)passes * RS_R));
        GB_CUDA(cudaMemsetAsync(hist, 0, (size_t)passes * RS_R * sizeof(unsigned long long), s));
        const int hist_blocks =
            (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)ctx->num_sms * 4, (n + 511) / 512));
        rs_hist_kernel<<<hist_blocks, 512, 0, s>>>(keys, n, plan, hist);
        note_launch();
    }
    rs_scan_kernel<<<1, RS_R, 0, s>>>(hist_in ? hist_in : hist, passes, portions, base);
    note_launch();
    GB_CUDA(cudaGetLastError());

    uint64_t *kc = keys, *ka = keys_alt;
    uint32_t *vc = vals, *va = vals_alt;
    const uint64_t tmo = timeout_ns();
    for (int p = 0; p < passes; ++p) {
        const int shift = plan.shift[p];
        const bool wide = plan.bits[p] == 9;
        for (int64_t q = 0; q < portions; ++q) {
            const int64_t pb = q * portion;
            const int64_t pc = std::min(portion, n - pb);
            const int ntiles = (int)((pc + RS_TILE - 1) / RS_TILE);
            GB_CUDA(cudaMemsetAsync(status, 0, (1 + (size_t)ntiles * (1 << plan.bits[p])) * sizeof(unsigned), s));
            const unsigned long long *bin = base + ((size_t)p * (portions + 1) + q) * RS_R;
            unsigned long long *bout = base + ((size_t)p * (portions + 1) + q + 1) * RS_R;
            if (has_vals && wide)
                rs_onesweep_kernel<true, 9><<<ntiles, RS_THREADS, dyn_smem, s>>>(
                    kc, ka, vc, va, pb, pc, shift, ntiles, bin, bout, status, ctx->status, tmo, n);
            else if (has_vals)
                rs_onesweep_kernel<true, 8><<<ntiles, RS_THREADS, dyn_smem, s>>>(
                    kc, ka, vc, va, pb, pc, shift, ntiles, bin, bout, status, ctx->status, tmo, n);
            else if (wide)
                rs_onesweep_kernel<false, 9><<<ntiles, RS_THREADS, dyn_smem, s>>>(
                    kc, ka, nullptr, nullptr, pb, pc, shift, ntiles, bin, bout, status, ctx->status,
                    tmo, n);
            else
                rs_onesweep_kernel<false, 8><<<ntiles, RS_THREADS, dyn_smem, s>>>(
                    kc, ka, nullptr, nullptr, pb, pc, shift, ntiles, bin, bout, status, ctx->status,
                    tmo, n);
            note_launch();
            GB_CUDA(cudaGetLastError());
        }
        std::swap(kc, ka);
        std::swap(vc, va);
    }
    *keys_out = kc;
    if (vals_out) *vals_out = vc;
    return GB_OK;
}

}  // namespace gb
