// Shared device helpers of the GB300 Graph500 library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gb300bfs.h"
#include "internal.h"

namespace gb {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Device status word: the first error a kernel records wins; nothing traps.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void record_error(DevStatus *st, int code, int where, long long detail)
{
    if (atomicCAS(&st->code, 0, code) == 0) {
        st->where = where;
        st->detail = detail;
    }
}

__device__ __forceinline__ int status_code(const DevStatus *st)
{
    return *(volatile const int *)&st->code;
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_volatile_u32(const unsigned *p)
{
    return *(volatile const unsigned *)p;
}

// ---------------------------------------------------------------------------
// Software grid barrier for cooperative (all-blocks-resident) launches.
// Arrivals only ever add to one counter: the k-th barrier of a launch is
// passed once the counter reaches base + k * gridDim.x, so no block has to
// reset anything and the last arrival frees the others directly.  Thread 0
// arrives with a release add (after __syncthreads, it publishes the block's
// writes) and waits with acquire loads.  Every wait is bounded by
// `timeout_ns` of the global timer: on expiry the block records
// GB_ERR_TIMEOUT, and every block leaves early once any block has recorded an
// error; grid_sync then returns false.
// ---------------------------------------------------------------------------
struct GridBarrier {
    unsigned count;
    unsigned pad;
};

__device__ __forceinline__ void red_release_add_u32(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// The counter value this launch starts from (a multiple of gridDim.x: every
// earlier launch on the same barrier passed all its barriers).  Call once at
// kernel entry, before the block's first grid_sync.
__device__ __forceinline__ unsigned grid_barrier_base(GridBarrier *b)
{
    __shared__ unsigned s_base;
    if (threadIdx.x == 0) s_base = (ld_acquire_u32(&b->count) / gridDim.x) * gridDim.x;
    __syncthreads();
    return s_base;
}

__device__ __forceinline__ bool grid_sync(GridBarrier *b, unsigned &target, DevStatus *st,
                                          uint64_t timeout_ns, int site)
{
    __shared__ int s_ok;
    target += gridDim.x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        red_release_add_u32(&b->count, 1u);
        uint64_t t0 = 0;
        unsigned spins = 0;
        while ((int)(ld_acquire_u32(&b->count) - target) < 0) {
            if (status_code(st) != 0) {
                ok = 0;
                break;
            }
            if ((++spins & 31u) == 0) {
                const uint64_t now = globaltimer_ns();
                if (t0 == 0) {
                    t0 = now;
                } else if (now - t0 > timeout_ns) {
                    record_error(st, GB_ERR_TIMEOUT, site, (long long)blockIdx.x);
                    ok = 0;
                    break;
                }
            }
            __nanosleep(32);
        }
        s_ok = ok && status_code(st) == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------------------
// Warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// inclusive prefix sum across the warp
template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v)
{
    const unsigned lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(kFull, v, o);
        if (lane >= (unsigned)o) v += t;
    }
    return v;
}

// Loads that bypass L1: data written by other blocks of the same kernel.
__device__ __forceinline__ unsigned ldcg_u32(const unsigned *p) { return __ldcg(p); }
__device__ __forceinline__ int ldcg_i32(const int *p) { return __ldcg(p); }
__device__ __forceinline__ unsigned long long ldcg_u64(const unsigned long long *p)
{
    return __ldcg(p);
}

// A hint (TMA bulk prefetch) that brings `bytes` bytes at p into L2; it
// neither waits nor changes any value.  p and bytes must be multiples of 16
// and the range must lie inside one allocation.
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

}  // namespace gb
