"""GPU parity of the device-side Graph500 validation (bfs_validate) and of
its TEPS counts.

The verdict code must equal the oracle's serial validator on every input,
valid trees and corrupted ones alike; the failing index must equal the one a
plain serial first-failure search (below) meets; reached, component and TEPS
edge counts must equal the oracle's.  Corrupted outputs are made on the host
and uploaded: the device kernels only read them (every value is range-checked
before it is used as an index).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2012_13548_gb300 as gb  # noqa: E402
from paper_2012_13548_gb300 import workloads as W  # noqa: E402
from tests.conftest import oracle_bfs, oracle_graph, roots_for  # noqa: E402

pytestmark = pytest.mark.gpu


def first_failure(off, col, root, parent, level):
    """(rule, index) of the first failure in the serial order: root range,
    rule 1, the vertices (7, 2), the vertices again (3, 4), the CSR entries
    (5, 6); (0, -1) if valid."""
    n = len(off) - 1
    if root < 0 or root >= n:
        return 7, root
    if parent[root] != root or level[root] != 0:
        return 1, root
    for v in range(n):
        if parent[v] < -1 or parent[v] >= n or level[v] < -1:
            return 7, v
        if (parent[v] == -1) != (level[v] == -1):
            return 2, v
    for v in range(n):
        if v == root or level[v] < 0:
            continue
        p = parent[v]
        if p not in set(col[off[v]:off[v + 1]].tolist()):
            return 3, v
        if level[p] != level[v] - 1:
            return 4, v
    for u in range(n):
        for e in range(off[u], off[u + 1]):
            v = col[e]
            if (level[u] < 0) != (level[v] < 0):
                return 5, e
            if level[u] >= 0 and abs(int(level[u]) - int(level[v])) > 1:
                return 6, e
    return 0, -1


def dev_graph(off, col):
    return gb.graph_from_csr(torch.as_tensor(off).cuda(), torch.as_tensor(col).cuda())


def check(G, off, col, root, parent, level, edges=None):
    parent = np.asarray(parent, dtype=np.int32)
    level = np.asarray(level, dtype=np.int32)
    res = gb.bfs_validate(G, root, torch.as_tensor(parent).cuda(), torch.as_tensor(level).cuda(),
                          None if edges is None else torch.as_tensor(edges).cuda())
    code_ref = oracle.validate(off, col, root, parent, level)
    code_bf, where_bf = first_failure(off, col, root, parent, level)
    assert code_bf == code_ref
    assert res["code"] == code_ref, (res, code_ref)
    assert res["where"] == where_bf, (res, where_bf)
    return res


@pytest.mark.parametrize("scale", [10, 14])
def test_valid_trees_and_counts_match_the_oracle(scale):
    e_ref, off, col = oracle_graph(scale)
    spec = W.GraphSpec(scale=scale)
    edges = gb.kron_generate(**spec.kron_args())
    G = gb.graph_build_csr(edges, scale)
    for canonical in (0, 1):
        gb.bfs_set_options(canonical_parents=canonical)
        for r in roots_for(scale, 6):
            parent, level = gb.bfs(G, r)
            res = gb.bfs_validate(G, r, parent, level, edges)
            _, lev_ref = oracle_bfs(scale, r)
            assert res["code"] == 0 and res["where"] == -1
            assert res["reached"] == int((lev_ref >= 0).sum())
            assert res["max_level"] == int(lev_ref.max())
            assert res["teps_edges"] == oracle.teps_edges(e_ref, lev_ref)
            assert res["component_edges"] == oracle.component_edges(off, lev_ref)
    gb.bfs_set_options(canonical_parents=0)
    # every row of a batched search
    rs = roots_for(scale, 8)
    P, L = gb.bfs_batch(G, rs)
    for i, r in enumerate(rs):
        res = gb.bfs_validate(G, r, P[i], L[i])
        assert res["code"] == 0 and res["teps_edges"] == -1
    G.free()


def test_every_rule_and_the_serial_precedence():
    _, off, col = oracle_graph(10)
    G = dev_graph(off, col)
    n = len(off) - 1
    r = roots_for(10, 1)[0]
    par0, lev0 = oracle_bfs(10, r)
    deg = np.diff(off)
    reached = np.nonzero((lev0 > 0))[0]
    rng = np.random.default_rng(3)

    def case(mut):
        p, lv = par0.copy(), lev0.copy()
        mut(p, lv)
        return check(G, off, col, r, p, lv)

    assert case(lambda p, lv: None)["code"] == 0
    nb = int(col[off[r]])
    assert case(lambda p, lv: p.__setitem__(r, nb))["code"] == 1
    assert case(lambda p, lv: lv.__setitem__(r, 1))["code"] == 1
    v = int(rng.choice(reached))
    assert case(lambda p, lv: p.__setitem__(v, -1))["code"] == 2
    iso = int(np.nonzero(deg == 0)[0][0])
    assert case(lambda p, lv: lv.__setitem__(iso, 2))["code"] == 2
    # a parent one level up that is not a neighbour
    for v in rng.permutation(reached):
        nbrs = set(col[off[v]:off[v + 1]].tolist())
        cands = [w for w in np.nonzero(lev0 == lev0[v] - 1)[0] if w not in nbrs]
        if cands:
            w = int(cands[0])
            assert case(lambda p, lv: p.__setitem__(int(v), w))["code"] == 3
            break
    # a neighbour on the same level as parent
    for v in rng.permutation(reached):
        same = [w for w in col[off[v]:off[v + 1]] if lev0[w] == lev0[v]]
        if same:
            w = int(same[0])
            assert case(lambda p, lv: p.__setitem__(int(v), w))["code"] == 4
            break
    # a leaf dropped from the tree: its edges now join reached and unreached
    children = np.bincount(par0[par0 >= 0], minlength=n)
    leaf = int([v for v in reached if children[v] == 0 or (children[v] == 1 and par0[v] == v)][0])

    def drop(p, lv):
        p[leaf] = -1
        lv[leaf] = -1
    assert case(drop)["code"] == 5
    assert case(lambda p, lv: p.__setitem__(int(reached[0]), n + 5))["code"] == 7
    assert case(lambda p, lv: lv.__setitem__(iso, -7))["code"] == 7
    assert case(lambda p, lv: p.__setitem__(iso, -2))["code"] == 7
    res = gb.bfs_validate(G, n, torch.as_tensor(par0).cuda(), torch.as_tensor(lev0).cuda())
    assert res["code"] == 7 and oracle.validate(off, col, n, par0, lev0) == 7
    # precedence: a later vertex-pass failure beats an earlier parent-pass one
    lo, hi = int(reached.min()), int(reached.max())

    def two(p, lv):
        p[lo] = p[r] if p[r] != lo and int(p[r]) not in set(col[off[lo]:off[lo + 1]].tolist()) else p[lo]
        p[hi] = -1
    assert case(two)["code"] == 2
    # many random corruptions at once
    for t in range(20):
        def many(p, lv, t=t):
            k = rng.integers(1, 6)
            for v in rng.integers(0, n, size=k):
                if rng.random() < 0.5:
                    p[v] = rng.integers(-3, n + 3)
                else:
                    lv[v] = rng.integers(-3, 12)
        case(many)
    G.free()


def test_rule_six_on_a_triangle():
    # triangle 0-1-2: from 0 both others are on level 1; the output below
    # claims the path 0-1-2, which passes rules 1-5 but not 6 on edge (0, 2)
    off = np.array([0, 2, 4, 6], dtype=np.int64)
    col = np.array([1, 2, 0, 2, 0, 1], dtype=np.int32)
    G = dev_graph(off, col)
    res = check(G, off, col, 0, [0, 0, 1], [0, 1, 2])
    assert res["code"] == 6 and res["where"] == 1
    assert check(G, off, col, 0, [0, 0, 0], [0, 1, 1])["code"] == 0
    G.free()


def test_random_small_graphs_all_roots():
    rng = np.random.default_rng(11)
    for trial in range(6):
        n = int(rng.integers(2, 120))
        e = rng.integers(0, n, size=(2, int(rng.integers(0, 3 * n)))).astype(np.int64)
        off, col = oracle.csr_build(e, max(1, (n - 1).bit_length()))
        off = off[: n + 1].copy()
        G = dev_graph(off, col)
        for root in range(n):
            parent, level = gb.bfs(G, root)
            res = gb.bfs_validate(G, root, parent, level)
            assert res["code"] == 0
            _, lev_ref = oracle.bfs(off, col, root)
            assert res["component_edges"] == oracle.component_edges(off, lev_ref)
        G.free()


def test_large_scale_trees_validate():
    scale = 20
    spec = W.GraphSpec(scale=scale)
    edges = gb.kron_generate(**spec.kron_args())
    G = gb.graph_build_csr(edges, scale)
    off, _ = G.csr()
    rs = [int(x) for x in W.select_roots(off.cpu().numpy(), 4, spec.seeds()[3])]
    for r in rs:
        parent, level = gb.bfs(G, r)
        res = gb.bfs_validate(G, r, parent, level, edges)
        assert res["code"] == 0
        lv = level.cpu()
        assert res["reached"] == int((lv >= 0).sum())
        assert res["teps_edges"] == int((level[edges[0]] >= 0).sum().item())
        # one corrupted entry is found at its index
        bad = parent.clone()
        v = int(torch.nonzero(level > 0)[-1])
        bad[v] = -1
        res = gb.bfs_validate(G, r, bad, level)
        assert res["code"] == 2 and res["where"] == v
    G.free()
