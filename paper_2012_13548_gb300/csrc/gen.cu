// Kronecker edge-list generator on the device (Sec. 2.1).
//
// #V = 2^scale, #E = edgefactor * #V.  Tuple e makes `scale` independent
// quadrant choices, one per bit level, from two SplitMix64 draws (Steele, Lea,
// Flood 2014) at counters 2(e*scale+k) and 2(e*scale+k)+1; a 53-bit draw is
// compared with integer thresholds floor(p * 2^53) so that the row bit is set
// with probability C+D and the column bit with B/(A+B) or D/(C+D).  Vertex
// numbers are then permuted (rank under (SplitMix64(seed_perm, v), v)) and the
// tuples shuffled (position j takes the tuple of rank j under
// (SplitMix64(seed_shuf, e), e)), both by the device radix sort.  Duplicates
// and self-loops stay in the list, as Sec. 2.1 requires.
#include "common.cuh"
#include "internal.h"

#include <string>

namespace gb {
namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void gen_hash_iota_kernel(int64_t count, uint64_t seed, uint64_t *__restrict__ keys,
                                     uint32_t *__restrict__ ids)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        keys[i] = splitmix64(seed, (uint64_t)i);
        ids[i] = (uint32_t)i;
    }
}

// Sec. 2.1 weight row: tuple j weighs (1 + the top 24 bits of
// SplitMix64(seed_w, j)) * 2^-24, a multiple of 2^-24 in (0, 1]; the integer
// is at most 2^24 and the scale a power of two, so the float is exact.
__global__ void gen_weights_kernel(int64_t m, uint64_t seed_w, float *__restrict__ w)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
        const uint32_t k = 1u + (uint32_t)(splitmix64(seed_w, (uint64_t)j) >> 40);
        w[j] = (float)k * 5.9604644775390625e-8f;  // 2^-24
    }
}

// pi[v] = rank of v: the sorted id list read as rank -> vertex, inverted.
__global__ void gen_perm_scatter_kernel(const uint32_t *__restrict__ sorted_ids, int64_t n,
                                        int32_t *__restrict__ pi, DevStatus *st)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        const uint32_t v = sorted_ids[r];
        if (v < n) pi[v] = (int32_t)r;
        else record_error(st, GB_ERR_RANGE, 40, r);
    }
}

// Tuple e from its counters: `scale` quadrant choices, bit k of the row and
// column ids from the draws at counters 2(e*scale+k) and 2(e*scale+k)+1.
__device__ __forceinline__ void kron_tuple(int scale, uint64_t e, uint64_t t_ab, uint64_t t_a,
                                           uint64_t t_c, uint64_t seed_gen, uint32_t &u,
                                           uint32_t &v)
{
    u = 0;
    v = 0;
    uint64_t ctr = 2ull * e * (uint64_t)scale;
    for (int k = 0; k < scale; ++k, ctr += 2) {
        const uint64_t x1 = splitmix64(seed_gen, ctr) >> 11;
        const uint64_t x2 = splitmix64(seed_gen, ctr + 1) >> 11;
        const uint32_t ii = x1 >= t_ab;
        const uint32_t jj = x2 >= (ii ? t_c : t_a);
        u |= ii << k;
        v |= jj << k;
    }
}

// Output position j: tuple order[j], generated from its counters and relabelled.
__global__ void __launch_bounds__(256) gen_edges_kernel(int scale, int64_t m, uint64_t t_ab,
                                                        uint64_t t_a, uint64_t t_c,
                                                        uint64_t seed_gen,
                                                        const uint32_t *__restrict__ order,
                                                        const int32_t *__restrict__ pi,
                                                        int64_t *__restrict__ edges, DevStatus *st)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
        const uint64_t e = order[j];
        if (e >= (uint64_t)m) {
            record_error(st, GB_ERR_RANGE, 41, j);
            continue;
        }
        uint32_t u, v;
        kron_tuple(scale, e, t_ab, t_a, t_c, seed_gen, u, v);
        edges[j] = pi[u];
        edges[m + j] = pi[v];
    }
}

// Kernel 1 fed straight from the generator: tuple e, relabelled, gives the two
// symmetric keys (u << S | v) and (v << S | u) at key positions 2e and 2e+1.
// The order of the tuples does not change the CSR, so the shuffle is skipped.
__global__ void __launch_bounds__(256) gen_keys_kernel(int scale, int64_t m, uint64_t t_ab,
                                                       uint64_t t_a, uint64_t t_c,
                                                       uint64_t seed_gen,
                                                       const int32_t *__restrict__ pi,
                                                       ulonglong2 *__restrict__ keys)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        uint32_t u, v;
        kron_tuple(scale, (uint64_t)e, t_ab, t_a, t_c, seed_gen, u, v);
        const uint64_t pu = (uint32_t)pi[u], pv = (uint32_t)pi[v];
        keys[e] = make_ulonglong2((pu << scale) | pv, (pv << scale) | pu);
    }
}

uint64_t threshold53(double p)
{
    const double two53 = 9007199254740992.0;
    if (!(p > 0.0)) return 0;  // also catches NaN from an empty quadrant pair
    return (uint64_t)(p * two53);
}

}  // namespace

namespace {

struct KronParams {
    int64_t n, m;
    uint64_t t_ab, t_a, t_c;
};

gb_status kron_params(int scale, int edgefactor, double a, double b, double c, const char *who,
                      KronParams &p)
{
    if (scale < 1 || scale > 30 || edgefactor < 1) {
        set_error(std::string(who) + ": need 1 <= scale <= 30, edgefactor >= 1");
        return GB_ERR_INVALID;
    }
    p.n = int64_t(1) << scale;
    p.m = p.n * edgefactor;
    if (p.m > (int64_t(1) << 32)) {
        set_error(std::string(who) + ": more than 2^32 tuples");
        return GB_ERR_RANGE;
    }
    const double d = 1.0 - a - b - c;
    p.t_ab = threshold53(a + b);
    p.t_a = threshold53(a / (a + b));
    p.t_c = threshold53(c / (c + d));
    return GB_OK;
}

// pi[v] = rank of v under (SplitMix64(seed_perm, v), v), by the radix sort;
// k0, k1, v0, v1 are scratch of at least n entries.
gb_status kron_perm(int64_t n, uint64_t seed_perm, uint64_t *k0, uint64_t *k1, uint32_t *v0,
                    uint32_t *v1, int32_t *pi, cudaStream_t s)
{
    Context *ctx = context();
    const int blocks = ctx->num_sms * 8;
    uint64_t *ks = nullptr;
    uint32_t *vs = nullptr;
    gen_hash_iota_kernel<<<blocks, 256, 0, s>>>(n, seed_perm, k0, v0);
    note_launch();
    GB_CUDA(cudaGetLastError());
    gb_status rc = radix_sort(k0, k1, v0, v1, n, 0, 64, &ks, &vs, s);
    if (rc != GB_OK) return rc;
    gen_perm_scatter_kernel<<<blocks, 256, 0, s>>>(vs, n, pi, ctx->status);
    note_launch();
    GB_CUDA(cudaGetLastError());
    return GB_OK;
}

}  // namespace

gb_status kron_generate_impl(int scale, int edgefactor, double a, double b, double c,
                             uint64_t seed_gen, uint64_t seed_perm, uint64_t seed_shuf,
                             int64_t *edges, cudaStream_t s)
{
    if (!edges) {
        set_error("kron_generate: edges == NULL");
        return GB_ERR_INVALID;
    }
    KronParams P;
    gb_status rc = kron_params(scale, edgefactor, a, b, c, "kron_generate", P);
    if (rc != GB_OK) return rc;
    const int64_t n = P.n, m = P.m;
    const uint64_t t_ab = P.t_ab, t_a = P.t_a, t_c = P.t_c;
    Context *ctx = context();
    if (!ctx) return GB_ERR_CUDA;
    const int blocks = ctx->num_sms * 8;
    // Vertex permutation.
    uint64_t *k0 = nullptr, *k1 = nullptr, *ks = nullptr;
    uint32_t *v0 = nullptr, *v1 = nullptr, *vs = nullptr;
    int32_t *pi = nullptr;
    Scratch tmp(s);
    GB_CUDA(tmp.alloc(&k0, (size_t)m));
    GB_CUDA(tmp.alloc(&k1, (size_t)m));
    GB_CUDA(tmp.alloc(&v0, (size_t)m));
    GB_CUDA(tmp.alloc(&v1, (size_t)m));
    GB_CUDA(tmp.alloc(&pi, (size_t)n));
    rc = kron_perm(n, seed_perm, k0, k1, v0, v1, pi, s);
    if (rc != GB_OK) return rc;
    // Edge shuffle order.
    gen_hash_iota_kernel<<<blocks, 256, 0, s>>>(m, seed_shuf, k0, v0);
    note_launch();
    GB_CUDA(cudaGetLastError());
    rc = radix_sort(k0, k1, v0, v1, m, 0, 64, &ks, &vs, s);
    if (rc != GB_OK) return rc;
    gen_edges_kernel<<<blocks, 256, 0, s>>>(scale, m, t_ab, t_a, t_c, seed_gen, vs, pi, edges,
                                            ctx->status);
    note_launch();
    GB_CUDA(cudaGetLastError());
    return GB_OK;
}

gb_status kron_keys_impl(int scale, int edgefactor, double a, double b, double c,
                         uint64_t seed_gen, uint64_t seed_perm, uint64_t *keys, cudaStream_t s)
{
    KronParams P;
    gb_status rc = kron_params(scale, edgefactor, a, b, c, "graph_generate_csr", P);
    if (rc != GB_OK) return rc;
    Context *ctx = context();
    if (!ctx) return GB_ERR_CUDA;
    uint64_t *k0 = nullptr, *k1 = nullptr;
    uint32_t *v0 = nullptr, *v1 = nullptr;
    int32_t *pi = nullptr;
    Scratch tmp(s);
    GB_CUDA(tmp.alloc(&k0, (size_t)P.n));
    GB_CUDA(tmp.alloc(&k1, (size_t)P.n));
    GB_CUDA(tmp.alloc(&v0, (size_t)P.n));
    GB_CUDA(tmp.alloc(&v1, (size_t)P.n));
    GB_CUDA(tmp.alloc(&pi, (size_t)P.n));
    rc = kron_perm(P.n, seed_perm, k0, k1, v0, v1, pi, s);
    if (rc != GB_OK) return rc;
    gen_keys_kernel<<<ctx->num_sms * 8, 256, 0, s>>>(scale, P.m, P.t_ab, P.t_a, P.t_c, seed_gen, pi,
                                                     reinterpret_cast<ulonglong2 *>(keys));
    note_launch();
    GB_CUDA(cudaGetLastError());
    return GB_OK;
}

gb_status kron_weights_impl(int64_t m, uint64_t seed_w, float *w, cudaStream_t s)
{
    Context *ctx = context();
    if (!ctx) return GB_ERR_CUDA;
    if (m == 0) return GB_OK;
    gen_weights_kernel<<<ctx->num_sms * 8, 256, 0, s>>>(m, seed_w, w);
    note_launch();
    GB_CUDA(cudaGetLastError());
    return GB_OK;
}

}  // namespace gb
