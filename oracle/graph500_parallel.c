/*
 * The paper's multicore method on the host CPU: the timed CPU baseline.
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY, like graph500_oracle.c beside it:
 * it may be called from tests/ and from bench.py's CPU legs (cpu_baseline and
 * the reference arm), and from nothing else.  It shares no code, header,
 * table or helper with the CUDA library and includes none of its files.
 *
 * Paper: "Graph500 from OCaml-Multicore Perspective" (arXiv 2012.13548).
 *
 *   gbp_bfs       Sec. 2.3.2, Algorithm "Parallel BFS": a level-synchronous
 *                 search in which the vertices of the current level and their
 *                 neighbours are processed in parallel, an unvisited
 *                 neighbour (level -1) getting level l+1 and joining the next
 *                 level; the next level starts only once the whole current
 *                 level is done (the synchronisation the section shows is
 *                 needed).  The paper parallelises both loops, over the
 *                 level's vertices and over each vertex's neighbours; here
 *                 the level's edges are split evenly among the threads, so a
 *                 vertex of huge degree is shared by all of them.  Where the
 *                 algorithm lets several threads set level(u) and enqueue u,
 *                 a compare-and-swap on level(u) lets exactly one thread
 *                 claim u, which also records the frontier vertex it came
 *                 from as parent(u) (any valid Graph500 tree).
 *   gbp_kron_csr  the graph of Sec. 2.1's Kronecker generator, built as the
 *                 CSR of Sec. 2.2 in parallel: tuples drawn in parallel
 *                 (identical to the serial oracle's, tuple by tuple),
 *                 relabelled by the same permutation, their two symmetric
 *                 keys sorted by a parallel radix sort (Sec. 4.2 proposes a
 *                 parallel sort for kernel 1), duplicates and self-loops
 *                 dropped.  The tuple shuffle of Sec. 2.1 only orders the
 *                 tuples, which a CSR does not see, so no edge list is made.
 *                 It also counts, per vertex, the tuples that start there
 *                 (the TEPS numerator of Sec. 4.3 sums them over the reached
 *                 vertices).
 *
 * Both are pinned to the serial oracle by tests (levels and CSR equal, trees
 * valid) before any timing is trusted.  Threads: OpenMP, as many as asked
 * (0 = all the runtime offers).
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GBP_OK 0
#define GBP_ERR_INVALID (-1)
#define GBP_ERR_NOMEM (-2)
#define GBP_ERR_RANGE (-5)

static int gbp_nthreads(int want)
{
    return want > 0 ? want : omp_get_max_threads();
}

int gbp_max_threads(void) { return omp_get_max_threads(); }

/* SplitMix64 (Steele, Lea, Flood 2014): output function of state
 * seed + (i + 1) * golden-ratio gamma. */
static inline uint64_t gbp_sm64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* ------------------------------------------------------------------------ */
/* Parallel LSD radix sort of uint64 keys by their low `bits` bits, 8 bits a  */
/* pass, optionally carrying uint32 values.  Each thread counts the digits of */
/* its contiguous block, the counts are scanned digit-major and thread-minor, */
/* and each thread scatters its block in order, so every pass is stable.     */
/* ------------------------------------------------------------------------ */
static int gbp_radix_sort(uint64_t **keys, uint64_t **alt, uint32_t **vals, uint32_t **valt,
                          int64_t n, int bits, int nth)
{
    const int passes = (bits + 7) / 8;
    int64_t *cnt = (int64_t *)malloc((size_t)nth * 256 * sizeof(int64_t));
    if (!cnt) return GBP_ERR_NOMEM;
    uint64_t *k = *keys, *kt = *alt;
    uint32_t *v = vals ? *vals : NULL, *vt = valt ? *valt : NULL;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        int used = nth;
#pragma omp parallel num_threads(nth)
        {
            const int t = omp_get_thread_num();
            const int T = omp_get_num_threads();
#pragma omp single
            used = T;
            const int64_t lo = n * t / T, hi = n * (t + 1) / T;
            int64_t h[256];
            memset(h, 0, sizeof(h));
            for (int64_t i = lo; i < hi; ++i) ++h[(k[i] >> shift) & 255u];
            memcpy(cnt + (size_t)t * 256, h, sizeof(h));
#pragma omp barrier
#pragma omp single
            {
                int64_t s = 0;
                for (int d = 0; d < 256; ++d)
                    for (int u = 0; u < used; ++u) {
                        const int64_t c = cnt[(size_t)u * 256 + d];
                        cnt[(size_t)u * 256 + d] = s;
                        s += c;
                    }
            }
            int64_t pos[256];
            memcpy(pos, cnt + (size_t)t * 256, sizeof(pos));
            if (v) {
                for (int64_t i = lo; i < hi; ++i) {
                    const int64_t o = pos[(k[i] >> shift) & 255u]++;
                    kt[o] = k[i];
                    vt[o] = v[i];
                }
            } else {
                for (int64_t i = lo; i < hi; ++i) kt[pos[(k[i] >> shift) & 255u]++] = k[i];
            }
        }
        uint64_t *sk = k; k = kt; kt = sk;
        uint32_t *sv = v; v = vt; vt = sv;
    }
    free(cnt);
    *keys = k;
    *alt = kt;
    if (vals) { *vals = v; *valt = vt; }
    return GBP_OK;
}

/* ------------------------------------------------------------------------ */
/* The CSR of the Kronecker graph (Sec. 2.1 generator, Sec. 2.2 CSR).        */
/* off: int64 [n+1]; col: int32 with room for 2m entries; starts: int64 [n]   */
/* (tuples whose start vertex is v, duplicates and self-loops included);     */
/* *nnz receives the columns used.  Thresholds floor(p * 2^53) for the row   */
/* bit (p = A+B) and the column bit (A/(A+B) after a 0 row bit, C/(C+D)      */
/* after a 1); tuple e, level k draws counters 2(e*scale+k) and +1.  The      */
/* permutation is the rank of v in ascending (SM64(seed_perm, v), v).        */
/* ------------------------------------------------------------------------ */
int gbp_kron_csr(int scale, int edgefactor, double a, double b, double c, uint64_t seed_gen,
                 uint64_t seed_perm, int threads, int64_t *off, int32_t *col, int64_t *starts,
                 int64_t *nnz)
{
    if (scale < 1 || scale > 30 || edgefactor < 1) return GBP_ERR_INVALID;
    const int nth = gbp_nthreads(threads);
    const int64_t n = (int64_t)1 << scale;
    const int64_t m = n * (int64_t)edgefactor;
    const int64_t nk = 2 * m;
    const double two53 = 9007199254740992.0;
    const double d = 1.0 - a - b - c;
    const uint64_t t_row = (uint64_t)((a + b) * two53);
    const uint64_t t_col0 = (uint64_t)((a / (a + b)) * two53);
    const uint64_t t_col1 = (uint64_t)((c / (c + d)) * two53);
    const uint64_t lowmask = ((uint64_t)1 << scale) - 1u;
    const uint64_t none = ((uint64_t)1 << (2 * scale)) - 1u;  /* above every real key */

    uint64_t *hk = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    uint64_t *hk2 = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    uint32_t *id = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint32_t *id2 = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint32_t *pi = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint64_t *key = (uint64_t *)malloc((size_t)nk * sizeof(uint64_t));
    uint64_t *key2 = (uint64_t *)malloc((size_t)nk * sizeof(uint64_t));
    int rc = GBP_ERR_NOMEM;
    if (!hk || !hk2 || !id || !id2 || !pi || !key || !key2) goto out;

    /* the vertex permutation: sort (hash, id) by hash; ids start ascending and
     * every pass is stable, so equal hashes would stay in id order */
#pragma omp parallel for num_threads(nth) schedule(static)
    for (int64_t v = 0; v < n; ++v) {
        hk[v] = gbp_sm64(seed_perm, (uint64_t)v);
        id[v] = (uint32_t)v;
        starts[v] = 0;
    }
    rc = gbp_radix_sort(&hk, &hk2, &id, &id2, n, 64, nth);
    if (rc != GBP_OK) goto out;
#pragma omp parallel for num_threads(nth) schedule(static)
    for (int64_t r = 0; r < n; ++r) pi[id[r]] = (uint32_t)r;

    /* every tuple, relabelled, gives its two symmetric keys (a self-loop two
     * keys above every real one, dropped after the sort) */
#pragma omp parallel for num_threads(nth) schedule(static, 4096)
    for (int64_t e = 0; e < m; ++e) {
        uint64_t u = 0, v = 0;
        for (int k = 0; k < scale; ++k) {
            const uint64_t ctr = 2u * ((uint64_t)e * (uint64_t)scale + (uint64_t)k);
            const uint64_t x1 = gbp_sm64(seed_gen, ctr) >> 11;
            const uint64_t x2 = gbp_sm64(seed_gen, ctr + 1u) >> 11;
            const uint64_t ii = x1 >= t_row;
            const uint64_t jj = x2 >= (ii ? t_col1 : t_col0);
            u |= ii << k;
            v |= jj << k;
        }
        const uint64_t pu = pi[u], pv = pi[v];
        __atomic_fetch_add(&starts[pu], 1, __ATOMIC_RELAXED);
        if (pu == pv) {
            key[2 * e] = none;
            key[2 * e + 1] = none;
        } else {
            key[2 * e] = (pu << scale) | pv;
            key[2 * e + 1] = (pv << scale) | pu;
        }
    }
    rc = gbp_radix_sort(&key, &key2, NULL, NULL, nk, 2 * scale, nth);
    if (rc != GBP_OK) goto out;

    /* distinct keys become the columns; a row's first key sets its offset and
     * the offsets of the empty rows before it */
    {
        int64_t *part = (int64_t *)calloc((size_t)nth + 1, sizeof(int64_t));
        if (!part) { rc = GBP_ERR_NOMEM; goto out; }
        int used = nth;
#pragma omp parallel num_threads(nth)
        {
            const int t = omp_get_thread_num();
            const int T = omp_get_num_threads();
#pragma omp single
            used = T;
            const int64_t lo = nk * t / T, hi = nk * (t + 1) / T;
            int64_t kept = 0;
            for (int64_t i = lo; i < hi; ++i)
                kept += key[i] != none && (i == 0 || key[i] != key[i - 1]);
            part[t + 1] = kept;
#pragma omp barrier
#pragma omp single
            for (int u = 0; u < used; ++u) part[u + 1] += part[u];
            int64_t pos = part[t];
            for (int64_t i = lo; i < hi; ++i) {
                const uint64_t ki = key[i];
                if (ki == none || (i > 0 && ki == key[i - 1])) continue;
                const int64_t row = (int64_t)(ki >> scale);
                const int64_t prev = i == 0 ? -1 : (key[i - 1] == none ? n : (int64_t)(key[i - 1] >> scale));
                for (int64_t r = prev + 1; r <= row; ++r) off[r] = pos;
                col[pos++] = (int32_t)(ki & lowmask);
            }
        }
        const int64_t total = part[used];
        free(part);
        /* rows after the last key (and every row of an empty graph) */
        int64_t last = -1;
        for (int64_t i = nk - 1; i >= 0; --i)
            if (key[i] != none) { last = (int64_t)(key[i] >> scale); break; }
        for (int64_t r = last + 1; r <= n; ++r) off[r] = total;
        *nnz = total;
    }
    rc = GBP_OK;
out:
    free(hk); free(hk2); free(id); free(id2); free(pi); free(key); free(key2);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.3.2, Algorithm "Parallel BFS" (see the top of the file).  Returns  */
/* the number of levels (max level + 1) or a negative error.                 */
/* ------------------------------------------------------------------------ */
int64_t gbp_bfs(const int64_t *off, const int32_t *col, int64_t n, int64_t root, int threads,
                int32_t *parent, int32_t *level)
{
    if (n < 1) return GBP_ERR_INVALID;
    if (root < 0 || root >= n) return GBP_ERR_RANGE;
    const int nth = gbp_nthreads(threads);
    int32_t *q = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *qn = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int64_t *dsum = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    int64_t *part = (int64_t *)calloc((size_t)nth + 1, sizeof(int64_t));
    int32_t **buf = (int32_t **)calloc((size_t)nth, sizeof(int32_t *));
    int64_t *cap = (int64_t *)calloc((size_t)nth, sizeof(int64_t));
    int64_t nlev = GBP_ERR_NOMEM;
    if (!q || !qn || !dsum || !part || !buf || !cap) goto out;

#pragma omp parallel for num_threads(nth) schedule(static)
    for (int64_t v = 0; v < n; ++v) {
        level[v] = -1;
        parent[v] = -1;
    }
    level[root] = 0;
    parent[root] = (int32_t)root;
    q[0] = (int32_t)root;
    int64_t qlen = 1;
    int32_t l = 0;
    int fail = 0;
    while (qlen > 0 && !fail) {
        /* the level's edges, numbered by a prefix sum of the frontier degrees */
        dsum[0] = 0;
        for (int64_t i = 0; i < qlen; ++i) dsum[i + 1] = dsum[i] + (off[q[i] + 1] - off[q[i]]);
        const int64_t total = dsum[qlen];
        int used = nth;
#pragma omp parallel num_threads(nth)
        {
            const int t = omp_get_thread_num();
            const int T = omp_get_num_threads();
#pragma omp single
            used = T;
            const int64_t e0 = total * t / T, e1 = total * (t + 1) / T;
            int64_t len = 0;
            if (e0 < e1) {
                /* the frontier vertex holding edge e0 */
                int64_t lo = 0, hi = qlen;
                while (hi - lo > 1) {
                    const int64_t mid = (lo + hi) / 2;
                    if (dsum[mid] <= e0) lo = mid; else hi = mid;
                }
                int64_t i = lo, e = e0;
                while (e < e1) {
                    const int32_t v = q[i];
                    const int64_t rs = off[v] + (e - dsum[i]);
                    const int64_t re = off[v] + (e1 < dsum[i + 1] ? e1 - dsum[i] : dsum[i + 1] - dsum[i]);
                    for (int64_t j = rs; j < re; ++j) {
                        const int32_t u = col[j];
                        int32_t expect = -1;
                        if (__atomic_load_n(&level[u], __ATOMIC_RELAXED) == -1 &&
                            __atomic_compare_exchange_n(&level[u], &expect, l + 1, 0, __ATOMIC_RELAXED,
                                                        __ATOMIC_RELAXED)) {
                            parent[u] = v;
                            if (len == cap[t]) {
                                const int64_t nc = cap[t] ? 2 * cap[t] : 4096;
                                int32_t *nb = (int32_t *)realloc(buf[t], (size_t)nc * sizeof(int32_t));
                                if (!nb) {
                                    __atomic_store_n(&fail, 1, __ATOMIC_RELAXED);
                                    break;
                                }
                                buf[t] = nb;
                                cap[t] = nc;
                            }
                            buf[t][len++] = u;
                        }
                    }
                    e += re - rs;
                    ++i;
                }
            }
            part[t + 1] = len;
#pragma omp barrier
#pragma omp single
            {
                part[0] = 0;
                for (int u = 0; u < used; ++u) part[u + 1] += part[u];
            }
            if (len) memcpy(qn + part[t], buf[t], (size_t)len * sizeof(int32_t));
        }
        qlen = part[used];
        int32_t *s = q; q = qn; qn = s;
        ++l;
    }
    nlev = fail ? GBP_ERR_NOMEM : (int64_t)l;
out:
    if (buf)
        for (int t = 0; t < nth; ++t) free(buf[t]);
    free(buf); free(cap); free(q); free(qn); free(dsum); free(part);
    return nlev;
}

/* TEPS numerator (Sec. 4.3) from per-vertex start counts: the tuples whose
 * start vertex was reached. */
int64_t gbp_teps_edges(const int64_t *starts, const int32_t *level, int64_t n, int threads)
{
    const int nth = gbp_nthreads(threads);
    int64_t s = 0;
#pragma omp parallel for num_threads(nth) reduction(+ : s) schedule(static)
    for (int64_t v = 0; v < n; ++v)
        if (level[v] >= 0) s += starts[v];
    return s;
}
