/*
 * Graph500 oracle: a plain, serial, obviously-correct CPU statement of what the
 * GPU path computes.  TEST INFRASTRUCTURE ONLY: it may be called from tests/,
 * from __graft_entry__.smoke() and from bench.py's cpu_baseline / reference arm,
 * and from nothing else.  It shares no code, header, table or helper with the
 * CUDA library and includes none of its files.
 *
 * Paper: "Graph500 from OCaml-Multicore Perspective" (arXiv 2012.13548).
 *   Sec. 2      Graph500 outline (Algorithm "Basic Outline of Graph500")
 *   Sec. 2.1    Kronecker edge list: #V = 2^scale, #E = #V * edgefactor,
 *               duplicates and self-loops kept, vertices permuted then
 *               edges shuffled
 *   Sec. 2.2    CSR: empty rows repeat the previous offset, the last row's end
 *               is stored (n+1 offsets)
 *   Sec. 2.3.1  Algorithm "Sequential BFS" (level array; the tree follows
 *               from the level array)
 *   Sec. 4.3    TEPS over 64 roots
 *
 * Readings of the paper taken here (each is also listed in the design notes):
 *   - the Kronecker initiator, its per-bit quadrant sampling and the random
 *     stream are not in the paper: quadrant probabilities A,B,C,D and the
 *     SplitMix64 counter generator (Steele, Lea, Flood, OOPSLA 2014) are
 *     used, with integer thresholds so that every implementation decides each
 *     bit identically;
 *   - the random vertex relabelling and the random tuple order of Sec. 2.1
 *     are read as sort-by-hash: ascending (SplitMix64(seed, id), id);
 *   - Algorithm "Sequential BFS" marks a vertex visited only when it is
 *     dequeued, so a vertex can be enqueued twice and get a too-large level
 *     (triangle r-a-b from r gives level(b)=2).  The oracle marks on enqueue,
 *     which is what Algorithm "Parallel BFS" does with its level(u) = -1 test;
 *   - "for all index in E" on the per-vertex arrays is read as "in V";
 *   - the parent array is built from the level array: parent(v) is the
 *     smallest-id neighbour one level up (the canonical BFS tree);
 *   - the weight row of the 3 x #E matrix (kernel 3 only; BFS ignores it)
 *     is drawn per output tuple j as (1 + (SM64(seed_w, j) >> 40)) * 2^-24:
 *     uniform on the 2^24 multiples of 2^-24 in (0, 1].  Strictly positive
 *     weights keep every tight-parent tree acyclic, and every path length is
 *     then a multiple of 2^-24 below 2^29, which fp64 holds exactly: the
 *     distances below are exact, with no rounding to agree on;
 *   - kernel 1 keeps, for a pair joined by several tuples, the smallest of
 *     their weights (a shortest path only ever uses the lightest copy);
 *   - Algorithm "Sequential SSSP" takes the vertex of Q with the least
 *     distance; among equal distances the oracle takes the smallest id, and
 *     it stops once that least distance is infinite (the vertices left are
 *     unreachable and no relaxation can change them);
 *   - besides that algorithm's prev array, the canonical SSSP tree is
 *     defined like the BFS one: parent(v) is the smallest-id neighbour u with
 *     dist(u) + w(u,v) = dist(v).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GBO_OK 0
#define GBO_ERR_INVALID (-1)
#define GBO_ERR_NOMEM (-2)
#define GBO_ERR_RANGE (-5)

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea, Flood 2014): the output function applied to the  */
/* i-th state of a generator started at `seed` with the golden-ratio gamma.  */
/* ------------------------------------------------------------------------ */
uint64_t gbo_sm64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Integer thresholds for the per-bit quadrant choice of the Kronecker
 * recursion (Sec. 2.1 generator; initiator A,B,C,D = 1-A-B-C):
 *   t[0] = floor((A+B) * 2^53)        row bit is 1 iff x1 >= t[0]
 *   t[1] = floor(A/(A+B) * 2^53)      given row bit 0, column bit is 1 iff x2 >= t[1]
 *   t[2] = floor(C/(C+D) * 2^53)      given row bit 1, column bit is 1 iff x2 >= t[2]
 * so P(row 0, col 0) = A, P(0,1) = B, P(1,0) = C, P(1,1) = D. */
void gbo_kron_thresholds(double a, double b, double c, uint64_t t[3])
{
    const double two53 = 9007199254740992.0;
    double d = 1.0 - a - b - c;
    t[0] = (uint64_t)((a + b) * two53);
    t[1] = (uint64_t)((a / (a + b)) * two53);
    t[2] = (uint64_t)((c / (c + d)) * two53);
}

/* Raw Kronecker tuples before the permutation and the shuffle.
 * Tuple e, bit level k in [0, scale): r1 = SM64(seed, 2(e*scale+k)),
 * r2 = SM64(seed, 2(e*scale+k)+1); x = r >> 11 (53 bits); the row bit and
 * column bit of level k follow the thresholds above. */
int gbo_kron_raw(int scale, int64_t m, double a, double b, double c,
                 uint64_t seed_gen, int64_t *u_out, int64_t *v_out)
{
    if (scale < 1 || scale > 30 || m < 0) return GBO_ERR_INVALID;
    uint64_t t[3];
    gbo_kron_thresholds(a, b, c, t);
    for (int64_t e = 0; e < m; ++e) {
        int64_t u = 0, v = 0;
        for (int k = 0; k < scale; ++k) {
            uint64_t ctr = 2u * ((uint64_t)e * (uint64_t)scale + (uint64_t)k);
            uint64_t x1 = gbo_sm64(seed_gen, ctr) >> 11;
            uint64_t x2 = gbo_sm64(seed_gen, ctr + 1u) >> 11;
            int ii = x1 >= t[0];
            int jj = x2 >= (ii ? t[2] : t[1]);
            u |= (int64_t)ii << k;
            v |= (int64_t)jj << k;
        }
        u_out[e] = u;
        v_out[e] = v;
    }
    return GBO_OK;
}

typedef struct { uint64_t h; int64_t id; } gbo_hid;

static int gbo_cmp_hid(const void *pa, const void *pb)
{
    const gbo_hid *x = (const gbo_hid *)pa, *y = (const gbo_hid *)pb;
    if (x->h != y->h) return x->h < y->h ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

/* order[j] = the id of rank j when ids 0..count-1 are sorted ascending by
 * (SM64(seed, id), id). */
int gbo_hash_order(int64_t count, uint64_t seed, int64_t *order)
{
    if (count < 0) return GBO_ERR_INVALID;
    gbo_hid *tmp = (gbo_hid *)malloc((size_t)(count > 0 ? count : 1) * sizeof(gbo_hid));
    if (!tmp) return GBO_ERR_NOMEM;
    for (int64_t i = 0; i < count; ++i) {
        tmp[i].h = gbo_sm64(seed, (uint64_t)i);
        tmp[i].id = i;
    }
    qsort(tmp, (size_t)count, sizeof(gbo_hid), gbo_cmp_hid);
    for (int64_t j = 0; j < count; ++j) order[j] = tmp[j].id;
    free(tmp);
    return GBO_OK;
}

/* Vertex permutation (Sec. 2.1: the generated vertex ids are relabelled at
 * random): pi[v] = rank of v in ascending (SM64(seed_perm, v), v). */
int gbo_vertex_perm(int scale, uint64_t seed_perm, int64_t *pi)
{
    if (scale < 1 || scale > 30) return GBO_ERR_INVALID;
    int64_t n = (int64_t)1 << scale;
    int64_t *order = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!order) return GBO_ERR_NOMEM;
    int rc = gbo_hash_order(n, seed_perm, order);
    if (rc == GBO_OK)
        for (int64_t r = 0; r < n; ++r) pi[order[r]] = r;
    free(order);
    return rc;
}

/* The full generator of Sec. 2.1: m = edgefactor * 2^scale tuples; raw
 * tuples, then vertex ids relabelled by pi, then the tuples shuffled so that
 * output position j holds relabelled tuple order[j], order ascending by
 * (SM64(seed_shuf, e), e).  edges is [2][m]: row 0 start, row 1 end. */
int gbo_kron_generate(int scale, int edgefactor, double a, double b, double c,
                      uint64_t seed_gen, uint64_t seed_perm, uint64_t seed_shuf,
                      int64_t *edges)
{
    if (scale < 1 || scale > 30 || edgefactor < 1) return GBO_ERR_INVALID;
    int64_t n = (int64_t)1 << scale;
    int64_t m = n * (int64_t)edgefactor;
    int64_t *u = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    int64_t *v = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    int64_t *pi = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *order = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    int rc = GBO_ERR_NOMEM;
    if (u && v && pi && order) {
        rc = gbo_kron_raw(scale, m, a, b, c, seed_gen, u, v);
        if (rc == GBO_OK) rc = gbo_vertex_perm(scale, seed_perm, pi);
        if (rc == GBO_OK) rc = gbo_hash_order(m, seed_shuf, order);
        if (rc == GBO_OK) {
            for (int64_t j = 0; j < m; ++j) {
                int64_t e = order[j];
                edges[j] = pi[u[e]];
                edges[m + j] = pi[v[e]];
            }
        }
    }
    free(u); free(v); free(pi); free(order);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Kernel 1 (Sec. 2.2): undirected CSR.  Row u is the ascending set of        */
/* v != u with (u,v) or (v,u) among the tuples; off has n+1 entries, an empty */
/* row repeats the previous offset and off[n] = nnz.                          */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t u, v; } gbo_pair;

static int gbo_cmp_pair(const void *pa, const void *pb)
{
    const gbo_pair *x = (const gbo_pair *)pa, *y = (const gbo_pair *)pb;
    if (x->u != y->u) return x->u < y->u ? -1 : 1;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;
    return 0;
}

/* col must hold 2*m entries; *nnz receives the entries used. */
int gbo_csr_build(const int64_t *edges, int64_t m, int scale,
                  int64_t *off, int32_t *col, int64_t *nnz)
{
    if (scale < 1 || scale > 30 || m < 0) return GBO_ERR_INVALID;
    int64_t n = (int64_t)1 << scale;
    gbo_pair *p = (gbo_pair *)malloc((size_t)(2 * m + 1) * sizeof(gbo_pair));
    if (!p) return GBO_ERR_NOMEM;
    int64_t cnt = 0;
    for (int64_t e = 0; e < m; ++e) {
        int64_t a = edges[e], b = edges[m + e];
        if (a < 0 || a >= n || b < 0 || b >= n) { free(p); return GBO_ERR_RANGE; }
        if (a == b) continue;              /* self-loops are ignored by K1 */
        p[cnt].u = a; p[cnt].v = b; ++cnt; /* the graph is undirected */
        p[cnt].u = b; p[cnt].v = a; ++cnt;
    }
    qsort(p, (size_t)cnt, sizeof(gbo_pair), gbo_cmp_pair);
    for (int64_t i = 0; i <= n; ++i) off[i] = 0;
    int64_t k = 0;
    for (int64_t i = 0; i < cnt; ++i) {
        if (i > 0 && p[i].u == p[i - 1].u && p[i].v == p[i - 1].v) continue; /* duplicate */
        col[k++] = (int32_t)p[i].v;
        off[p[i].u + 1] += 1;               /* degree of row u */
    }
    for (int64_t i = 0; i < n; ++i) off[i + 1] += off[i]; /* empty rows repeat */
    *nnz = k;
    free(p);
    return GBO_OK;
}

/* ------------------------------------------------------------------------ */
/* Kernel 2 (Sec. 2.3.1): queue BFS.  level(v) = hop distance from root, -1   */
/* if unreachable.  A vertex is marked when it is enqueued.  The BFS tree is  */
/* then read from the level array: parent(v) = the smallest-id neighbour u    */
/* with level(u) = level(v) - 1; parent(root) = root; -1 if unreached.        */
/* Returns the number of levels (max level + 1) or a negative error.         */
/* ------------------------------------------------------------------------ */
int64_t gbo_bfs(const int64_t *off, const int32_t *col, int64_t n, int64_t root,
                int32_t *parent, int32_t *level)
{
    if (n < 1) return GBO_ERR_INVALID;
    if (root < 0 || root >= n) return GBO_ERR_RANGE;
    int64_t *queue = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!queue) return GBO_ERR_NOMEM;
    for (int64_t i = 0; i < n; ++i) { level[i] = -1; parent[i] = -1; }
    int64_t head = 0, tail = 0, maxlev = 0;
    level[root] = 0;
    queue[tail++] = root;
    while (head < tail) {
        int64_t node = queue[head++];
        for (int64_t e = off[node]; e < off[node + 1]; ++e) {
            int64_t u = col[e];
            if (level[u] == -1) {
                level[u] = level[node] + 1;
                if (level[u] > maxlev) maxlev = level[u];
                queue[tail++] = u;
            }
        }
    }
    free(queue);
    for (int64_t v = 0; v < n; ++v) {
        if (level[v] < 0) continue;
        if (v == root) { parent[v] = (int32_t)root; continue; }
        for (int64_t e = off[v]; e < off[v + 1]; ++e) {
            int64_t u = col[e];
            if (level[u] == level[v] - 1 && (parent[v] < 0 || u < parent[v]))
                parent[v] = (int32_t)u;
        }
    }
    return maxlev + 1;
}

/* ------------------------------------------------------------------------ */
/* Graph500 result validation (the benchmark's rules, cited by the paper as  */
/* its reference [5]).  0 = valid, otherwise the first rule that failed:      */
/*   1  parent(root) != root or level(root) != 0                              */
/*   2  parent(v) = -1 and level(v) != -1, or the reverse                     */
/*   3  reached v != root whose parent is not a neighbour                      */
/*   4  reached v != root with level(parent(v)) != level(v) - 1               */
/*   5  a graph edge with exactly one reached endpoint                        */
/*   6  a graph edge whose endpoint levels differ by more than one            */
/*   7  a parent or level value out of range                                  */
/* Rules 1-4 make every tree path strictly decrease in level down to the     */
/* root (so the tree is acyclic and spans exactly the reached set); with      */
/* rules 5-6 the levels are the BFS distances.                                */
/* ------------------------------------------------------------------------ */
int gbo_validate(const int64_t *off, const int32_t *col, int64_t n, int64_t root,
                 const int32_t *parent, const int32_t *level)
{
    if (root < 0 || root >= n) return 7;
    if (parent[root] != root || level[root] != 0) return 1;
    for (int64_t v = 0; v < n; ++v) {
        if (parent[v] < -1 || parent[v] >= n || level[v] < -1) return 7;
        if ((parent[v] == -1) != (level[v] == -1)) return 2;
    }
    for (int64_t v = 0; v < n; ++v) {
        if (v == root || level[v] < 0) continue;
        int64_t p = parent[v];
        int found = 0;
        for (int64_t e = off[v]; e < off[v + 1]; ++e)
            if (col[e] == p) { found = 1; break; }
        if (!found) return 3;
        if (level[p] != level[v] - 1) return 4;
    }
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
            int64_t v = col[e];
            if ((level[u] < 0) != (level[v] < 0)) return 5;
            if (level[u] >= 0) {
                int64_t d = (int64_t)level[u] - level[v];
                if (d > 1 || d < -1) return 6;
            }
        }
    }
    return 0;
}

/* TEPS numerator (Sec. 4.3 / Graph500): the input tuples whose start vertex
 * was reached, duplicates and self-loops included. */
int64_t gbo_teps_edges(const int64_t *edges, int64_t m, const int32_t *level)
{
    int64_t cnt = 0;
    for (int64_t e = 0; e < m; ++e)
        if (level[edges[e]] >= 0) ++cnt;
    return cnt;
}

/* Undirected simple edges inside the reached component: half the CSR
 * entries of reached rows. */
int64_t gbo_component_edges(const int64_t *off, int64_t n, const int32_t *level)
{
    int64_t s = 0;
    for (int64_t v = 0; v < n; ++v)
        if (level[v] >= 0) s += off[v + 1] - off[v];
    return s / 2;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1: the weight row of the 3 x #E tuple matrix (see the readings at   */
/* the top): w[j] = (1 + (SM64(seed_w, j) >> 40)) / 2^24 for output tuple j.  */
/* ------------------------------------------------------------------------ */
int gbo_kron_weights(int64_t m, uint64_t seed_w, double *w)
{
    if (m < 0) return GBO_ERR_INVALID;
    for (int64_t j = 0; j < m; ++j)
        w[j] = (double)(1u + (gbo_sm64(seed_w, (uint64_t)j) >> 40)) / 16777216.0;
    return GBO_OK;
}

/* ------------------------------------------------------------------------ */
/* Kernel 1 with the weight row (Sec. 2.2 CSR; the graph is weighted, Sec. 2): */
/* off and col as gbo_csr_build; wgt[k] is the smallest weight among the      */
/* tuples joining the pair of entry k, in either direction.                  */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t u, v; double w; } gbo_wpair;

static int gbo_cmp_wpair(const void *pa, const void *pb)
{
    const gbo_wpair *x = (const gbo_wpair *)pa, *y = (const gbo_wpair *)pb;
    if (x->u != y->u) return x->u < y->u ? -1 : 1;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;
    if (x->w != y->w) return x->w < y->w ? -1 : 1;
    return 0;
}

int gbo_csr_build_weighted(const int64_t *edges, const double *w, int64_t m, int scale,
                           int64_t *off, int32_t *col, double *wgt, int64_t *nnz)
{
    if (scale < 1 || scale > 30 || m < 0) return GBO_ERR_INVALID;
    int64_t n = (int64_t)1 << scale;
    gbo_wpair *p = (gbo_wpair *)malloc((size_t)(2 * m + 1) * sizeof(gbo_wpair));
    if (!p) return GBO_ERR_NOMEM;
    int64_t cnt = 0;
    for (int64_t e = 0; e < m; ++e) {
        int64_t a = edges[e], b = edges[m + e];
        if (a < 0 || a >= n || b < 0 || b >= n) { free(p); return GBO_ERR_RANGE; }
        if (!(w[e] > 0.0 && w[e] <= 1.0)) { free(p); return GBO_ERR_RANGE; }
        if (a == b) continue;
        p[cnt].u = a; p[cnt].v = b; p[cnt].w = w[e]; ++cnt;
        p[cnt].u = b; p[cnt].v = a; p[cnt].w = w[e]; ++cnt;
    }
    /* sorted by (u, v, w): the first entry of each (u, v) run has its least weight */
    qsort(p, (size_t)cnt, sizeof(gbo_wpair), gbo_cmp_wpair);
    for (int64_t i = 0; i <= n; ++i) off[i] = 0;
    int64_t k = 0;
    for (int64_t i = 0; i < cnt; ++i) {
        if (i > 0 && p[i].u == p[i - 1].u && p[i].v == p[i - 1].v) continue;
        col[k] = (int32_t)p[i].v;
        wgt[k] = p[i].w;
        ++k;
        off[p[i].u + 1] += 1;
    }
    for (int64_t i = 0; i < n; ++i) off[i + 1] += off[i];
    *nnz = k;
    free(p);
    return GBO_OK;
}

/* ------------------------------------------------------------------------ */
/* Kernel 3 (Sec. 2.4, Algorithm "Sequential SSSP", Dijkstra): dist[v] = the  */
/* least total weight of a path from root (INFINITY if none), prev[v] = the  */
/* vertex whose relaxation last lowered dist[v] (-1 for the root and for      */
/* unreached vertices, as the algorithm initialises it).  Q is kept in a      */
/* binary heap of (dist, id) entries; an entry whose vertex has left Q or     */
/* whose distance is out of date is skipped when it reaches the top, so the   */
/* vertex taken is the one of least (dist, id) in Q.                          */
/* Returns the number of vertices taken from Q (the reached ones).           */
/* ------------------------------------------------------------------------ */
typedef struct { double d; int64_t v; } gbo_hent;

static int gbo_hless(const gbo_hent *x, const gbo_hent *y)
{
    return x->d < y->d || (x->d == y->d && x->v < y->v);
}

int64_t gbo_sssp(const int64_t *off, const int32_t *col, const double *wgt, int64_t n,
                 int64_t root, double *dist, int32_t *prev)
{
    if (n < 1) return GBO_ERR_INVALID;
    if (root < 0 || root >= n) return GBO_ERR_RANGE;
    int64_t cap = off[n] + 2, hn = 0, taken = 0;
    gbo_hent *h = (gbo_hent *)malloc((size_t)cap * sizeof(gbo_hent));
    unsigned char *inq = (unsigned char *)malloc((size_t)n);
    if (!h || !inq) { free(h); free(inq); return GBO_ERR_NOMEM; }
    for (int64_t v = 0; v < n; ++v) { dist[v] = INFINITY; prev[v] = -1; inq[v] = 1; }
    dist[root] = 0.0;
    h[hn].d = 0.0; h[hn].v = root; ++hn;
    while (hn > 0) {
        gbo_hent top = h[0];
        /* pop: move the last entry to the top and sift it down */
        h[0] = h[--hn];
        for (int64_t i = 0;;) {
            int64_t l = 2 * i + 1, r = l + 1, b = i;
            if (l < hn && gbo_hless(&h[l], &h[b])) b = l;
            if (r < hn && gbo_hless(&h[r], &h[b])) b = r;
            if (b == i) break;
            gbo_hent t = h[i]; h[i] = h[b]; h[b] = t;
            i = b;
        }
        int64_t u = top.v;
        if (!inq[u] || top.d != dist[u]) continue;  /* left Q already, or out of date */
        inq[u] = 0;
        ++taken;
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
            int64_t v = col[e];
            if (!inq[v]) continue;                    /* v in Q and v in Adj[u] */
            double alt = dist[u] + wgt[e];
            if (alt < dist[v]) {
                dist[v] = alt;
                prev[v] = (int32_t)u;
                if (hn == cap) {                      /* cannot happen: one push per lowering */
                    free(h); free(inq);
                    return GBO_ERR_NOMEM;
                }
                /* push (alt, v) and sift it up */
                int64_t i = hn++;
                h[i].d = alt; h[i].v = v;
                while (i > 0) {
                    int64_t pa = (i - 1) / 2;
                    if (!gbo_hless(&h[i], &h[pa])) break;
                    gbo_hent t = h[i]; h[i] = h[pa]; h[pa] = t;
                    i = pa;
                }
            }
        }
    }
    free(h);
    free(inq);
    return taken;
}

/* The canonical SSSP tree of a distance array: parent(root) = root,
 * parent(v) = the smallest-id neighbour u with dist(u) + w(u,v) = dist(v),
 * -1 for unreached v. */
int gbo_sssp_tree(const int64_t *off, const int32_t *col, const double *wgt, int64_t n,
                  int64_t root, const double *dist, int32_t *parent)
{
    if (n < 1) return GBO_ERR_INVALID;
    if (root < 0 || root >= n) return GBO_ERR_RANGE;
    for (int64_t v = 0; v < n; ++v) {
        parent[v] = -1;
        if (v == root) { parent[v] = (int32_t)root; continue; }
        if (isinf(dist[v])) continue;
        for (int64_t e = off[v]; e < off[v + 1]; ++e) {
            int64_t u = col[e];
            if (dist[u] + wgt[e] == dist[v] && (parent[v] < 0 || u < parent[v]))
                parent[v] = (int32_t)u;
        }
    }
    return GBO_OK;
}

/* ------------------------------------------------------------------------ */
/* Kernel 3 result validation (Graph500's SSSP rules, the benchmark the       */
/* paper follows).  0 = valid, otherwise the first rule that failed:          */
/*   1  parent(root) != root or dist(root) != 0                               */
/*   2  parent(v) = -1 and dist(v) finite, or the reverse                     */
/*   3  reached v != root whose parent is not a neighbour                      */
/*   4  reached v != root with dist(v) != dist(parent) + w(parent, v)         */
/*   5  a graph edge with exactly one reached endpoint                        */
/*   6  a graph edge (u, v) with dist(v) > dist(u) + w(u, v)                   */
/*   7  a parent out of range, or a distance negative or NaN                  */
/* With positive weights rule 4 makes distances fall strictly along parent   */
/* links, so the tree is acyclic and ends at the root; with rule 6 every      */
/* distance is at most any path's length, so they are the shortest ones.     */
/* ------------------------------------------------------------------------ */
int gbo_sssp_validate(const int64_t *off, const int32_t *col, const double *wgt, int64_t n,
                      int64_t root, const int32_t *parent, const double *dist)
{
    if (root < 0 || root >= n) return 7;
    for (int64_t v = 0; v < n; ++v)
        if (parent[v] < -1 || parent[v] >= n || isnan(dist[v]) || dist[v] < 0.0) return 7;
    if (parent[root] != root || dist[root] != 0.0) return 1;
    for (int64_t v = 0; v < n; ++v)
        if ((parent[v] == -1) != (isinf(dist[v]) != 0)) return 2;
    for (int64_t v = 0; v < n; ++v) {
        if (v == root || parent[v] < 0) continue;
        int64_t p = parent[v], found = -1;
        for (int64_t e = off[v]; e < off[v + 1]; ++e)
            if (col[e] == p) { found = e; break; }
        if (found < 0) return 3;
        if (dist[p] + wgt[found] != dist[v]) return 4;
    }
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
            int64_t v = col[e];
            if (isinf(dist[u]) != isinf(dist[v])) return 5;
            if (!isinf(dist[u]) && dist[v] > dist[u] + wgt[e]) return 6;
        }
    }
    return 0;
}
