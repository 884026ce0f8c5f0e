"""Pins of the paper's multicore method (oracle/parallel.py, OpenMP), the timed
CPU baseline: before its times are reported it must compute what the serial
oracle computes.

* Algorithm "Parallel BFS" (Sec. 2.3.2): levels equal to the serial queue BFS
  (itself pinned in test_oracle.py) on the hand fixtures, closed forms and
  Kronecker graphs, at 1, 3 and 8 threads; its parents (the claiming frontier
  vertex) pass the Graph500 validator; the TEPS numerator from per-vertex
  start counts equals the oracle's count over the tuples.
* The parallel Kronecker CSR (Sec. 2.1, 2.2): offsets and columns equal to
  the oracle's build of the oracle's tuples, bit for bit, at every thread
  count, for the workload recipe and for other initiators and edgefactors;
  the start counts equal a bincount of the tuples' start row.
"""
import numpy as np
import pytest

import oracle
import oracle.parallel as P
from paper_2012_13548_gb300 import workloads as W
from tests.golden import load_hand_graphs

THREADS = [1, 3, 8]


@pytest.mark.parametrize("g", load_hand_graphs(), ids=lambda g: g["name"])
def test_parallel_bfs_hand_fixtures(g):
    scale = max(1, (g["n"] - 1).bit_length())
    off, col = oracle.csr_build(g["edges"], scale)
    n = g["n"]
    off = np.ascontiguousarray(off[: n + 1])
    for th in THREADS:
        parent, level, nl = P.bfs(off, col, g["root"], threads=th)
        assert np.array_equal(level, g["levels"]), (g["name"], th)
        assert nl == int(level.max()) + 1
        assert oracle.validate(off, col, g["root"], parent, level) == 0, (g["name"], th)


@pytest.mark.parametrize("n", [2, 7, 64, 1000])
def test_parallel_bfs_closed_forms(n):
    # path from one end: level i; cycle: min(i, n - i); star from a leaf: 2
    path = np.stack([np.arange(n - 1), np.arange(1, n)]).astype(np.int64)
    cyc = np.stack([np.arange(n), (np.arange(n) + 1) % n]).astype(np.int64)
    scale = max(1, (n - 1).bit_length())
    for edges, want in [(path, np.arange(n)), (cyc, np.minimum(np.arange(n), n - np.arange(n)))]:
        if n < 3 and edges is cyc:
            continue
        off, col = oracle.csr_build(edges, scale)
        off = np.ascontiguousarray(off[: n + 1])
        for th in THREADS:
            _, level, _ = P.bfs(off, col, 0, threads=th)
            assert np.array_equal(level, want.astype(np.int32)), (n, th)


@pytest.mark.parametrize("scale", [1, 2, 5, 8, 10, 12, 14, 16])
def test_parallel_kron_csr_equals_the_oracle(scale):
    spec = W.GraphSpec(scale=scale)
    kw = spec.kron_args()
    e = oracle.kron_generate(**kw)
    off_ref, col_ref = oracle.csr_build(e, scale)
    starts_ref = np.bincount(e[0], minlength=spec.n)
    for th in THREADS:
        off, col, starts = P.kron_csr(**kw, threads=th)
        assert np.array_equal(off, off_ref), th
        assert np.array_equal(col, col_ref), th
        assert np.array_equal(starts, starts_ref), th


def test_parallel_kron_csr_other_initiators_and_edgefactors():
    for (a, b, c, ef, scale) in [(0.25, 0.25, 0.25, 1, 9), (0.45, 0.15, 0.15, 3, 11),
                                 (1.0, 0.0, 0.0, 2, 5), (0.0, 0.0, 0.0, 2, 5)]:
        kw = dict(scale=scale, edgefactor=ef, a=a, b=b, c=c, seed_gen=11, seed_perm=12, seed_shuf=13)
        e = oracle.kron_generate(**kw)
        off_ref, col_ref = oracle.csr_build(e, scale)
        off, col, starts = P.kron_csr(**kw, threads=4)
        assert np.array_equal(off, off_ref) and np.array_equal(col, col_ref), (a, b, c, ef)
        assert np.array_equal(starts, np.bincount(e[0], minlength=1 << scale))


@pytest.mark.parametrize("scale", [10, 14, 16])
def test_parallel_bfs_on_kronecker_graphs(scale):
    spec = W.GraphSpec(scale=scale)
    kw = spec.kron_args()
    e = oracle.kron_generate(**kw)
    off, col, starts = P.kron_csr(**kw)
    roots = W.select_roots(off, 6, spec.seeds()[3])
    for r in [int(x) for x in roots]:
        _, level_ref = oracle.bfs(off, col, r)
        for th in THREADS:
            parent, level, nl = P.bfs(off, col, r, threads=th)
            assert np.array_equal(level, level_ref), (scale, r, th)
            assert oracle.validate(off, col, r, parent, level) == 0
            assert P.teps_edges(starts, level) == oracle.teps_edges(e, level)
    # an isolated vertex as root reaches only itself
    iso = int(np.nonzero(np.diff(off) == 0)[0][0])
    parent, level, nl = P.bfs(off, col, iso, threads=4)
    assert nl == 1 and int((level >= 0).sum()) == 1 and parent[iso] == iso


def test_parallel_bfs_rejects_bad_roots():
    off = np.array([0, 1, 2], dtype=np.int64)
    col = np.array([1, 0], dtype=np.int32)
    for bad in (-1, 2):
        with pytest.raises(RuntimeError):
            P.bfs(off, col, bad)
