"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: each checks it against a
published test vector, a hand-worked fixture, a closed form, a brute force on
tiny inputs, or an invariant that a plausible slip (a dropped term, a swapped
index or comparison, a transposed operand) would break.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from tests.golden import load_hand_graphs
from paper_2012_13548_gb300 import workloads as W

HAND = load_hand_graphs()


# --------------------------------------------------------------------------
# SplitMix64 (Steele, Lea, Flood 2014)
# --------------------------------------------------------------------------

def test_sm64_published_vectors():
    # splitmix64 started from state 0: its first three outputs as published with
    # the generator (state advanced by the golden gamma before each output).
    assert oracle.sm64(0, 0) == 0xE220A8397B1DCDAF
    assert oracle.sm64(0, 1) == 0x6E789E6AA1B965F4
    assert oracle.sm64(0, 2) == 0x06C45D188009454F


def test_sm64_counter_and_seed_are_one_stream():
    # counter i of seed s is the (i+1)-th state of one stream: seed s + gamma
    # continues the stream of seed s one step later.
    g = 0x9E3779B97F4A7C15
    for i in range(5):
        assert oracle.sm64(7, i + 1) == oracle.sm64((7 + g) % 2**64, i)


# --------------------------------------------------------------------------
# Kronecker generator (Sec. 2.1)
# --------------------------------------------------------------------------

def _bits(x, scale):
    return ((x[:, None] >> np.arange(scale)) & 1).astype(np.int64)


def test_kron_quadrant_frequencies():
    # P(row bit)=C+D, P(col bit)=B+D and the four quadrant frequencies A,B,C,D,
    # each within 5 sigma of a binomial over scale*m samples.
    scale, m = 16, 1 << 16
    u, v = oracle.kron_raw(scale, m, W.A, W.B, W.C, 12345)
    bu, bv = _bits(u, scale).ravel(), _bits(v, scale).ravel()
    N = bu.size
    D = 1 - W.A - W.B - W.C
    for got, p in [((bu == 0) & (bv == 0), W.A), ((bu == 0) & (bv == 1), W.B),
                   ((bu == 1) & (bv == 0), W.C), ((bu == 1) & (bv == 1), D),
                   (bu == 1, W.C + D), (bv == 1, W.B + D)]:
        sigma = math.sqrt(p * (1 - p) / N)
        assert abs(got.mean() - p) < 5 * sigma, (got.mean(), p)


def test_kron_degenerate_initiators():
    # A = 1: every tuple is (0, 0).  D = 1: every tuple is (n-1, n-1).
    u, v = oracle.kron_raw(6, 500, 1.0, 0.0, 0.0, 9)
    assert (u == 0).all() and (v == 0).all()
    u, v = oracle.kron_raw(6, 500, 0.0, 0.0, 0.0, 9)
    assert (u == 63).all() and (v == 63).all()
    # A=B=C=D=1/4: endpoints uniform over [0, n): chi-square on 16 cells
    u, v = oracle.kron_raw(4, 1 << 16, 0.25, 0.25, 0.25, 3)
    for x in (u, v):
        cnt = np.bincount(x, minlength=16)
        exp = x.size / 16
        chi2 = ((cnt - exp) ** 2 / exp).sum()
        assert chi2 < 60, chi2   # 15 dof; p < 1e-6 above 60


def test_kron_levels_and_tuples_draw_distinct_counters():
    # Each (tuple, level) pair uses its own counters: bits of neighbouring
    # levels and of neighbouring tuples are uncorrelated (a counter laid out as
    # e + k instead of e*scale + k would make them identical).
    scale, m = 12, 1 << 15
    u, v = oracle.kron_raw(scale, m, 0.25, 0.25, 0.25, 77)
    bu = _bits(u, scale).astype(float)
    bv = _bits(v, scale).astype(float)
    for a, b in [(bu[:-1, 1:], bu[1:, :-1]), (bu[:, 1:], bu[:, :-1]), (bu, bv),
                 (bu[:-1], bu[1:])]:
        c = np.corrcoef(a.ravel(), b.ravel())[0, 1]
        assert abs(c) < 0.02, c


def test_hash_order_is_the_sorted_hash_order():
    # order lists ids by ascending (SplitMix64(seed, id), id); numpy's lexsort
    # over hashes computed one by one gives the same list.
    seed, count = 99, 3000
    o = oracle.hash_order(count, seed)
    h = np.array([oracle.sm64(seed, i) for i in range(count)], dtype=np.uint64)
    ref = np.lexsort((np.arange(count), h))
    assert np.array_equal(o, ref)


def test_vertex_perm_is_rank_not_inverse():
    scale, seed = 9, 5
    pi = oracle.vertex_perm(scale, seed)
    n = 1 << scale
    assert np.array_equal(np.sort(pi), np.arange(n))          # a bijection
    h = np.array([oracle.sm64(seed, v) for v in range(n)], dtype=np.uint64)
    # pi[v] = rank of v: the vertex of smallest hash maps to 0
    assert pi[int(np.argmin(h))] == 0
    assert pi[int(np.argmax(h))] == n - 1
    assert all(h[a] < h[b] for a, b in zip(np.argsort(pi)[:-1], np.argsort(pi)[1:]))


def test_generator_counts_and_composition():
    spec = W.GraphSpec(scale=8)
    kw = spec.kron_args()
    e = oracle.kron_generate(**kw)
    assert e.shape == (2, 16 * 256)                             # #E = 16 * 2^scale
    assert e.min() >= 0 and e.max() < 256
    u, v = oracle.kron_raw(8, spec.m, W.A, W.B, W.C, kw["seed_gen"])
    pi = oracle.vertex_perm(8, kw["seed_perm"])
    # relabel first, then shuffle: position j holds relabelled tuple of rank j
    h = np.array([oracle.sm64(kw["seed_shuf"], i) for i in range(spec.m)], dtype=np.uint64)
    order = np.lexsort((np.arange(spec.m), h))
    assert np.array_equal(e[0], pi[u][order])
    assert np.array_equal(e[1], pi[v][order])
    # duplicates and self-loops are present in the list handed to kernel 1
    assert (e[0] == e[1]).any()
    pairs = set()
    dup = False
    for a, b in e.T:
        dup |= (a, b) in pairs
        pairs.add((a, b))
    assert dup


# --------------------------------------------------------------------------
# Kernel 1: CSR (Sec. 2.2)
# --------------------------------------------------------------------------

def _brute_csr(edges, n):
    rows = [set() for _ in range(n)]
    for a, b in edges.T:
        if a != b:
            rows[a].add(int(b))
            rows[b].add(int(a))
    off = [0]
    col = []
    for r in rows:
        col += sorted(r)
        off.append(len(col))
    return np.array(off, dtype=np.int64), np.array(col, dtype=np.int32)


@pytest.mark.parametrize("g", [g for g in HAND if "off" in g], ids=lambda g: g["name"])
def test_csr_hand_fixtures(g):
    off, col = oracle.csr_build(g["edges"], max(1, (g["n"] - 1).bit_length()))
    n = g["n"]
    assert np.array_equal(off[: n + 1], g["off"])
    assert np.array_equal(col, g["col"])


def test_csr_matches_set_brute_force():
    rng = np.random.default_rng(1)
    for trial in range(30):
        scale = int(rng.integers(1, 7))
        n = 1 << scale
        m = int(rng.integers(0, 4 * n))
        e = rng.integers(0, n, size=(2, m)).astype(np.int64)
        off, col = oracle.csr_build(e, scale)
        boff, bcol = _brute_csr(e, n)
        assert np.array_equal(off, boff) and np.array_equal(col, bcol), trial


def test_csr_invariants_and_shuffle_invariance():
    spec = W.GraphSpec(scale=10)
    e = oracle.kron_generate(**spec.kron_args())
    off, col = oracle.csr_build(e, 10)
    n = spec.n
    assert off[0] == 0 and off[-1] == col.size and col.size % 2 == 0
    assert (np.diff(off) >= 0).all()
    rows = np.repeat(np.arange(n), np.diff(off))
    assert (rows != col).all()                                   # no self-loops
    same_row = rows[1:] == rows[:-1]
    assert (col[1:][same_row] > col[:-1][same_row]).all()        # strictly ascending
    fwd = set(zip(rows.tolist(), col.tolist()))
    assert all((b, a) in fwd for a, b in fwd)                    # symmetric
    # the CSR does not depend on tuple order or multiplicity
    perm = np.random.default_rng(2).permutation(e.shape[1])
    off2, col2 = oracle.csr_build(np.ascontiguousarray(e[:, perm]), 10)
    off3, col3 = oracle.csr_build(np.concatenate([e, e[::-1]], axis=1), 10)
    assert np.array_equal(off, off2) and np.array_equal(col, col2)
    assert np.array_equal(off, off3) and np.array_equal(col, col3)


def test_csr_rejects_out_of_range():
    with pytest.raises(RuntimeError):
        oracle.csr_build(np.array([[0, 1], [1, 4]], dtype=np.int64), 2)


# --------------------------------------------------------------------------
# Kernel 2: BFS (Sec. 2.3.1)
# --------------------------------------------------------------------------

def _csr_of(g):
    return _brute_csr(g["edges"], g["n"])


@pytest.mark.parametrize("g", HAND, ids=lambda g: g["name"])
def test_bfs_hand_fixtures(g):
    off, col = _csr_of(g)
    parent, level = oracle.bfs(off, col, g["root"])
    assert np.array_equal(level, g["levels"])
    assert np.array_equal(parent, g["parents"])
    assert oracle.validate(off, col, g["root"], parent, level) == 0
    if "teps" in g:
        assert oracle.teps_edges(g["edges"], level) == g["teps"]


@pytest.mark.parametrize("n", [1, 2, 5, 17])
def test_bfs_closed_forms(n):
    # path: level i; cycle: min(i, n-i); complete graph: 1
    path = np.array([np.arange(n - 1), np.arange(1, n)], dtype=np.int64)
    off, col = _brute_csr(path, n)
    _, lev = oracle.bfs(off, col, 0)
    assert np.array_equal(lev, np.arange(n))
    if n >= 3:
        cyc = np.array([np.arange(n), (np.arange(n) + 1) % n], dtype=np.int64)
        off, col = _brute_csr(cyc, n)
        _, lev = oracle.bfs(off, col, 0)
        i = np.arange(n)
        assert np.array_equal(lev, np.minimum(i, n - i))
    kn = np.array(list(itertools.combinations(range(n), 2)), dtype=np.int64).reshape(-1, 2).T
    off, col = _brute_csr(kn, n)
    par, lev = oracle.bfs(off, col, n - 1)
    exp = np.ones(n, dtype=np.int32)
    exp[n - 1] = 0
    assert np.array_equal(lev, exp)
    assert (par == n - 1).all()


def _brute_levels(n, edges, root):
    """Distances by repeated relaxation over the adjacency matrix."""
    adj = np.zeros((n, n), dtype=bool)
    for a, b in edges.T:
        if a != b:
            adj[a, b] = adj[b, a] = True
    INF = 10 ** 9
    d = np.full(n, INF)
    d[root] = 0
    for _ in range(n):
        cand = np.where(adj, d[None, :] + 1, INF).min(axis=1)
        nd = np.minimum(d, cand)
        if np.array_equal(nd, d):
            break
        d = nd
    lev = np.where(d >= INF, -1, d).astype(np.int32)
    par = np.full(n, -1, dtype=np.int32)
    for v in range(n):
        if v == root:
            par[v] = root
        elif lev[v] > 0:
            par[v] = min(u for u in range(n) if adj[v, u] and lev[u] == lev[v] - 1)
    return par, lev


def test_bfs_matches_matrix_relaxation():
    rng = np.random.default_rng(7)
    for trial in range(40):
        n = int(rng.integers(1, 65))
        m = int(rng.integers(0, 3 * n))
        e = rng.integers(0, n, size=(2, m)).astype(np.int64)
        off, col = _brute_csr(e, n)
        for root in sorted(set([0, n - 1, int(rng.integers(0, n))])):
            par, lev = oracle.bfs(off, col, root)
            bpar, blev = _brute_levels(n, e, root)
            assert np.array_equal(lev, blev), (trial, root)
            assert np.array_equal(par, bpar), (trial, root)


def test_bfs_rejects_bad_root():
    off, col = _brute_csr(np.array([[0], [1]], dtype=np.int64), 2)
    with pytest.raises(RuntimeError):
        oracle.bfs(off, col, 2)
    with pytest.raises(RuntimeError):
        oracle.bfs(off, col, -1)


# --------------------------------------------------------------------------
# Validator (Graph500 rules) and the TEPS count (Sec. 4.3)
# --------------------------------------------------------------------------

def _kron10():
    spec = W.GraphSpec(scale=10)
    e = oracle.kron_generate(**spec.kron_args())
    off, col = oracle.csr_build(e, 10)
    root = int(W.select_roots(off, 1, spec.seeds()[3])[0])
    par, lev = oracle.bfs(off, col, root)
    return e, off, col, root, par, lev


def test_validator_accepts_any_valid_tree():
    e, off, col, root, par, lev = _kron10()
    assert oracle.validate(off, col, root, par, lev) == 0
    # a non-canonical but valid tree: the largest-id neighbour one level up
    alt = par.copy()
    for v in range(off.size - 1):
        if lev[v] > 0:
            nb = col[off[v]:off[v + 1]]
            alt[v] = nb[lev[nb] == lev[v] - 1].max()
    assert oracle.validate(off, col, root, alt, lev) == 0


def test_validator_rejects_planted_mistakes():
    e, off, col, root, par, lev = _kron10()
    reached = np.nonzero(lev > 1)[0]
    v = int(reached[0])
    cases = {}
    p = par.copy(); p[root] = int(col[off[root]]); cases[1] = (p, lev)          # root not own parent
    l2 = lev.copy(); l2[v] = -1; cases[2] = (par, l2)                           # parent set, level -1
    p = par.copy()
    non_nb = next(u for u in range(off.size - 1)
                  if u != v and u not in set(col[off[v]:off[v + 1]].tolist()))
    p[v] = non_nb; cases[3] = (p, lev)                                          # parent not a neighbour
    l3 = lev.copy(); l3[v] += 1; cases[4] = (par, l3)                           # wrong level
    unreached = np.nonzero(lev < 0)[0]
    # missed vertex: drop a reached leaf (no children) from the tree
    children = set(par[lev > 0].tolist())
    leaf = next(int(x) for x in np.nonzero(lev > 0)[0] if int(x) not in children)
    p = par.copy(); l5 = lev.copy(); p[leaf] = -1; l5[leaf] = -1; cases[5] = (p, l5)
    for rule, (p, l) in cases.items():
        assert oracle.validate(off, col, root, p, l) == rule, rule
    # a cycle among two reached vertices with consistent-looking levels fails
    a = int(np.nonzero(lev == 2)[0][0])
    p = par.copy(); p[int(par[a])] = a
    assert oracle.validate(off, col, root, p, lev) != 0
    assert unreached.size >= 0


def test_validator_catches_a_level_jump():
    # a path 0-1-2-3 with levels claiming 3 sits at level 1 through a non-edge
    off, col = _brute_csr(np.array([[0, 1, 2], [1, 2, 3]], dtype=np.int64), 4)
    par = np.array([0, 0, 1, 0], dtype=np.int32)
    lev = np.array([0, 1, 2, 1], dtype=np.int32)
    assert oracle.validate(off, col, 0, par, lev) == 3
    par = np.array([0, 0, 1, 2], dtype=np.int32)
    lev = np.array([0, 1, 2, 4], dtype=np.int32)
    assert oracle.validate(off, col, 0, par, lev) == 4


def test_teps_counts_component_tuples():
    e, off, col, root, par, lev = _kron10()
    m_r = oracle.teps_edges(e, lev)
    # tuples are counted with multiplicity and self-loops, by start vertex
    assert m_r == int((lev[e[0]] >= 0).sum())
    # the deduplicated count is half the CSR entries of reached rows
    assert oracle.component_edges(off, lev) * 2 == int(np.diff(off)[lev >= 0].sum())
    assert 0 < oracle.component_edges(off, lev) <= m_r


# --------------------------------------------------------------------------
# Kernel 3 (Sec. 2.4): the weight row, the weighted CSR, Dijkstra
# --------------------------------------------------------------------------

def test_weight_row_grid_range_and_uniformity():
    m = 200_000
    w = oracle.kron_weights(m, 12345)
    k = w * 2.0**24
    assert np.all(k == np.round(k)) and k.min() >= 1 and k.max() <= 2**24
    assert abs(w.mean() - 0.5) < 0.005
    counts = np.histogram(w, bins=16, range=(0.0, 1.0))[0]
    assert np.all(np.abs(counts - m / 16) < 0.05 * m / 16)
    assert not np.array_equal(w[:1000], oracle.kron_weights(1000, 12346))
    # the first weight of seed 0 from the published first SplitMix64 output
    # 0xE220A8397B1DCDAF: its top 24 bits, plus one, in units of 2^-24
    assert oracle.kron_weights(1, 0)[0] == (1 + 0xE220A8) / 2.0**24


def test_weighted_csr_keeps_the_least_weight_of_each_pair():
    rng = np.random.default_rng(5)
    for scale in [1, 2, 4, 6]:
        n = 1 << scale
        for m in [0, 1, 9, 5 * n]:
            e = rng.integers(0, n, size=(2, m)).astype(np.int64)
            w = rng.integers(1, 9, size=m) / 8.0
            off, col, wgt = oracle.csr_build_weighted(e, w, scale)
            off0, col0 = oracle.csr_build(e, scale)
            assert np.array_equal(off, off0) and np.array_equal(col, col0)
            best = {}
            for (a, b), x in zip(e.T.tolist(), w.tolist()):
                if a != b:
                    for key in ((a, b), (b, a)):
                        best[key] = min(best.get(key, 2.0), x)
            got = {(u, int(col[j])): float(wgt[j])
                   for u in range(n) for j in range(off[u], off[u + 1])}
            assert got == best


def test_weighted_csr_rejects_bad_weights_and_endpoints():
    e = np.array([[0, 1], [1, 2]], dtype=np.int64)
    for bad in ([0.5, 0.0], [0.5, 1.5], [0.5, float("nan")], [-0.25, 0.5]):
        with pytest.raises(RuntimeError):
            oracle.csr_build_weighted(e, np.array(bad), 2)
    with pytest.raises(RuntimeError):
        oracle.csr_build_weighted(np.array([[0], [4]]), np.array([0.5]), 2)


def test_sssp_hand_worked_diamond_with_a_tie():
    # 0-1 (1/2), 0-2 (1/4), 1-3 (1/4), 2-3 (1/2), 3-4 (1/8); 5 isolated.
    # Algorithm "Sequential SSSP": take 0 (dist 1 = 1/2, dist 2 = 1/4), take 2
    # (dist 3 = 3/4 by 2), take 1 (1/2 + 1/4 is not < 3/4: prev 3 stays 2),
    # take 3 (dist 4 = 7/8).  Both 1 and 2 are tight for 3: the canonical
    # tree takes 1.
    e = np.array([[0, 0, 1, 2, 3], [1, 2, 3, 3, 4]], dtype=np.int64)
    w = np.array([0.5, 0.25, 0.25, 0.5, 0.125])
    off, col, wgt = oracle.csr_build_weighted(e, w, 3)
    dist, prev = oracle.sssp(off, col, wgt, 0)
    inf = float("inf")
    assert dist.tolist() == [0.0, 0.5, 0.25, 0.75, 0.875, inf, inf, inf]
    assert prev.tolist() == [-1, 0, 0, 2, 3, -1, -1, -1]
    tree = oracle.sssp_tree(off, col, wgt, 0, dist)
    assert tree.tolist() == [0, 0, 0, 1, 3, -1, -1, -1]
    assert oracle.sssp_validate(off, col, wgt, 0, tree, dist) == 0


def test_sssp_path_closed_form():
    rng = np.random.default_rng(8)
    k = 200
    w = rng.integers(1, 2**24 + 1, size=k - 1) / 2.0**24
    e = np.stack([np.arange(k - 1), np.arange(1, k)]).astype(np.int64)
    off, col, wgt = oracle.csr_build_weighted(e, w, 8)
    dist, prev = oracle.sssp(off, col, wgt, 0)
    expect = np.concatenate([[0.0], np.cumsum(w)])
    assert np.array_equal(dist[:k], expect)          # exact: multiples of 2^-24
    assert np.all(np.isinf(dist[k:]))
    assert prev[1:k].tolist() == list(range(k - 1))
    # from the far end the distances are the suffix sums
    d2, _ = oracle.sssp(off, col, wgt, k - 1)
    assert np.array_equal(d2[:k], expect[-1] - expect)


def test_sssp_unit_weights_are_bfs_levels():
    spec = W.GraphSpec(scale=9)
    e = oracle.kron_generate(**spec.kron_args())
    w = np.ones(e.shape[1])
    off, col, wgt = oracle.csr_build_weighted(e, w, 9)
    for root in [int(np.argmax(np.diff(off))), 3, 100]:
        parent_b, level = oracle.bfs(off, col, root)
        dist, _ = oracle.sssp(off, col, wgt, root)
        reached = level >= 0
        assert np.array_equal(dist[reached], level[reached].astype(np.float64))
        assert np.all(np.isinf(dist[~reached]))
        assert np.array_equal(oracle.sssp_tree(off, col, wgt, root, dist), parent_b)


def _brute_force_distances(n, edges, w, root):
    adj = {}
    for (a, b), x in zip(edges.T.tolist(), w.tolist()):
        if a != b:
            adj.setdefault(a, []).append((b, x))
            adj.setdefault(b, []).append((a, x))
    best = [math.inf] * n
    best[root] = 0.0

    def walk(u, d, seen):
        for v, x in adj.get(u, []):
            if v not in seen:
                best[v] = min(best[v], d + x)
                walk(v, d + x, seen | {v})

    walk(root, 0.0, {root})
    return np.array(best)


def test_sssp_matches_all_simple_paths_on_tiny_graphs():
    rng = np.random.default_rng(21)
    for _ in range(60):
        n = int(rng.integers(2, 8))
        m = int(rng.integers(0, 14))
        e = rng.integers(0, n, size=(2, m)).astype(np.int64)
        w = rng.integers(1, 2**24 + 1, size=m) / 2.0**24
        off, col, wgt = oracle.csr_build_weighted(e, w, 3)
        root = int(rng.integers(0, n))
        dist, prev = oracle.sssp(off, col, wgt, root)
        assert np.array_equal(dist[:n], _brute_force_distances(n, e, w, root))
        assert np.all(np.isinf(dist[n:]))
        p = prev.copy()
        p[root] = root
        assert oracle.sssp_validate(off, col, wgt, root, p, dist) == 0
        assert oracle.sssp_validate(off, col, wgt, root,
                                    oracle.sssp_tree(off, col, wgt, root, dist), dist) == 0


def test_sssp_matches_scipy_dijkstra():
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    sparse = pytest.importorskip("scipy.sparse")
    rng = np.random.default_rng(34)
    for n, m in [(300, 900), (500, 600), (256, 4000)]:
        e = rng.integers(0, n, size=(2, m)).astype(np.int64)
        w = rng.integers(1, 2**24 + 1, size=m) / 2.0**24
        dense = np.full((n, n), np.inf)
        keep = e[0] != e[1]
        np.minimum.at(dense, (e[0][keep], e[1][keep]), w[keep])
        np.minimum.at(dense, (e[1][keep], e[0][keep]), w[keep])
        dense[np.isinf(dense)] = 0.0                    # no edge
        ref = csgraph.dijkstra(sparse.csr_matrix(dense), directed=True, indices=[0, 7])
        scale = max(1, (n - 1).bit_length())
        off, col, wgt = oracle.csr_build_weighted(e, w, scale)
        for i, root in enumerate([0, 7]):
            dist, _ = oracle.sssp(off, col, wgt, root)
            assert np.array_equal(dist[:n], ref[i])


def test_sssp_validator_rejects_planted_mistakes():
    spec = W.GraphSpec(scale=9)
    e = oracle.kron_generate(**spec.kron_args())
    w = oracle.kron_weights(e.shape[1], 77)
    off, col, wgt = oracle.csr_build_weighted(e, w, 9)
    root = int(np.argmax(np.diff(off)))
    dist, _ = oracle.sssp(off, col, wgt, root)
    tree = oracle.sssp_tree(off, col, wgt, root, dist)
    assert oracle.sssp_validate(off, col, wgt, root, tree, dist) == 0
    reached = np.flatnonzero(np.isfinite(dist))
    isolated = np.flatnonzero(np.diff(off) == 0)
    children = np.bincount(tree[tree >= 0], minlength=tree.size)
    # a leaf of the tree with a neighbour that is not tight for it
    v = next(int(x) for x in reached if x != root and children[x] == 0 and any(
        dist[col[j]] + wgt[j] > dist[x] for j in range(off[x], off[x + 1])))

    def check(rule, p=None, d=None):
        assert oracle.sssp_validate(off, col, wgt, root, tree if p is None else p,
                                    dist if d is None else d) == rule

    d = dist.copy(); d[root] = 2.0**-24; check(1, d=d)
    p = tree.copy(); p[root] = tree[v]; check(1, p=p)
    p = tree.copy(); p[v] = -1; check(2, p=p)
    non_nb = next(u for u in reached if u != v and u not in col[off[v]:off[v + 1]])
    p = tree.copy(); p[v] = non_nb; check(3, p=p)
    d = dist.copy(); d[v] += 2.0**-24; check(4, d=d)
    # v hung from a longer path: its tree edge is consistent, an edge is not
    j = next(j for j in range(off[v], off[v + 1]) if dist[col[j]] + wgt[j] > dist[v])
    p = tree.copy(); p[v] = col[j]
    d = dist.copy(); d[v] = dist[col[j]] + wgt[j]
    check(6, p=p, d=d)
    # an isolated vertex claimed as reached from a reached one
    x = int(isolated[0])
    p = tree.copy(); p[x] = root
    d = dist.copy(); d[x] = 1.0
    check(3, p=p, d=d)
    d = dist.copy(); d[v] = -1.0; check(7, d=d)
    p = tree.copy(); p[v] = tree.size; check(7, p=p)


def test_sssp_rejects_bad_root():
    off = np.array([0, 1, 2], dtype=np.int64)
    col = np.array([1, 0], dtype=np.int32)
    wgt = np.array([0.5, 0.5])
    with pytest.raises(RuntimeError):
        oracle.sssp(off, col, wgt, 2)
    with pytest.raises(RuntimeError):
        oracle.sssp(off, col, wgt, -1)
