"""Full-size checks that need no oracle run: at SCALE 24 and 26 the CSR must
be exactly the set of distinct symmetrised non-loop input tuples (computed
here with torch's own sort), which checks the chained multi-portion path the
radix sort takes above 2^28 keys; at SCALE 24 (and SCALE 26 when
GB_TEST_S26=1) the CSR must satisfy the Sec. 2.2 invariants and every BFS
result must pass the Graph500 rules, which together force the levels to be
the exact hop distances.  At SCALE 22 (the kernel-3 bench size) every
shortest-path result must be tight along its tree and relaxed over every
edge, which forces the exact distances.  The properties are computed here
with plain torch tensor operations, independently of the library."""
import os

import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2012_13548_gb300 as gb  # noqa: E402
from paper_2012_13548_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

SCALES = [24] + ([26] if os.environ.get("GB_TEST_S26") == "1" else [])


def csr_properties(off, col, n):
    assert off.numel() == n + 1 and int(off[0]) == 0 and int(off[-1]) == col.numel()
    deg = off[1:] - off[:-1]
    assert bool((deg >= 0).all())
    assert int(col.min()) >= 0 and int(col.max()) < n
    rows = torch.repeat_interleave(torch.arange(n, device=col.device, dtype=torch.int32), deg)
    assert bool((rows != col).all()), "self-loop in the CSR"
    same = rows[1:] == rows[:-1]
    assert bool((col[1:][same] > col[:-1][same]).all()), "row not strictly ascending"
    key = rows.to(torch.int64) * n + col.to(torch.int64)
    rkey = col.to(torch.int64) * n + rows.to(torch.int64)
    pos = torch.searchsorted(key, rkey)
    assert bool((key[pos.clamp(max=key.numel() - 1)] == rkey).all()), "CSR not symmetric"
    return rows, key


def tree_properties(off, col, rows, key, n, root, parent, level):
    assert int(level[root]) == 0 and int(parent[root]) == root
    assert bool(((parent == -1) == (level == -1)).all())
    lr, lc = level[rows.long()], level[col.long()]
    assert bool(((lr >= 0) == (lc >= 0)).all()), "edge leaves the reached set"
    assert bool(((lr - lc).abs()[lr >= 0] <= 1).all()), "edge spans two levels"
    v = torch.nonzero(level > 0).flatten()
    p = parent[v].long()
    assert bool((level[p] == level[v] - 1).all()), "parent not one level up"
    pk = v * n + p
    pos = torch.searchsorted(key, pk).clamp(max=key.numel() - 1)
    assert bool((key[pos] == pk).all()), "parent is not a neighbour"


def tuple_key_set(edges, n):
    """Sorted distinct keys row * n + col of the symmetrised input tuples
    without self-loops: what the CSR of Sec. 2.2 must hold, from torch.unique."""
    keep = edges[0] != edges[1]
    a, b = edges[0][keep], edges[1][keep]
    del keep
    tk = torch.cat([a * n + b, b * n + a])
    del a, b
    out = torch.unique(tk, sorted=True)
    del tk
    return out


@pytest.mark.parametrize("scale", [24, 26])
def test_full_size_csr_is_the_tuple_set(scale):
    # above 2^28 keys (kernel 1 from SCALE 24, the SCALE 26 generator's
    # shuffle) the radix sort chains several portions; a dropped or doubled
    # portion changes this set
    spec = W.GraphSpec(scale=scale)
    n = spec.n
    edges = gb.kron_generate(**spec.kron_args())
    assert int(edges.min()) >= 0 and int(edges.max()) < n
    want = tuple_key_set(edges, n)
    g = gb.graph_build_csr(edges, scale)
    off, col = g.csr()
    assert g.nnz == want.numel()
    deg = off[1:] - off[:-1]
    rows = torch.repeat_interleave(torch.arange(n, device=col.device, dtype=torch.int64), deg)
    assert torch.equal(rows * n + col.to(torch.int64), want), "CSR differs from the tuple set"
    del rows, deg
    g.free()
    # the fused generate-and-build path (no edge list) gives the same graph
    g = gb.graph_generate_csr(**spec.kron_args())
    off2, col2 = g.csr()
    assert g.nnz == want.numel()
    deg = off2[1:] - off2[:-1]
    rows = torch.repeat_interleave(torch.arange(n, device=col2.device, dtype=torch.int64), deg)
    assert torch.equal(rows * n + col2.to(torch.int64), want), "fused CSR differs from the tuple set"
    del rows, deg
    g.free()
    del want, edges
    torch.cuda.empty_cache()
    gb.gb_device_status()


@pytest.mark.parametrize("scale", SCALES)
def test_full_size_csr_and_bfs_properties(scale):
    spec = W.GraphSpec(scale=scale)
    edges = gb.kron_generate(**spec.kron_args())
    e0 = edges[0].clone()
    g = gb.graph_build_csr(edges, scale)
    del edges
    torch.cuda.empty_cache()
    off, col = g.csr()
    n = g.n
    rows, key = csr_properties(off, col, n)
    roots = W.select_roots(off.cpu().numpy(), 4, spec.seeds()[3])
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    for canonical in (0, 1):
        gb.bfs_set_options(canonical_parents=canonical)
        for r in roots:
            gb.bfs(g, int(r), parent, level)
            gb.gb_device_status()
            tree_properties(off, col, rows, key, n, int(r), parent, level)
            st = gb.bfs_last_stats()
            assert st["reached"] == int((level >= 0).sum())
    gb.bfs_set_options(canonical_parents=0)
    # the multi-source rows equal the single-source levels
    P, L = gb.bfs_batch(g, [int(r) for r in roots])
    for i, r in enumerate(roots):
        gb.bfs(g, int(r), parent, level)
        assert torch.equal(L[i], level)
        tree_properties(off, col, rows, key, n, int(r), P[i], L[i])
    gb.gb_device_status()
    del e0


def test_full_size_sssp_properties():
    scale = 22
    spec = W.GraphSpec(scale=scale)
    edges = gb.kron_generate(**spec.kron_args())
    w = gb.kron_weights(edges.shape[1], spec.seed_weight())
    g = gb.graph_build_csr_weighted(edges, w, scale)
    off, col = g.csr()
    n = g.n
    rows, key = csr_properties(off, col, n)
    wt = g.weights().to(torch.float64) * 2.0 ** -24
    # each entry's weight is the least weight of the tuples joining its pair
    keep = edges[0] != edges[1]
    tk = torch.cat([edges[0][keep] * n + edges[1][keep], edges[1][keep] * n + edges[0][keep]])
    tw = torch.cat([w[keep], w[keep]]).to(torch.float64)
    least = torch.full((key.numel(),), 2.0, dtype=torch.float64, device="cuda")
    least.scatter_reduce_(0, torch.searchsorted(key, tk), tw, reduce="amin")
    assert torch.equal(least, wt)
    del tk, tw, least
    roots = W.select_roots(off.cpu().numpy(), 3, spec.seeds()[3])
    for canonical in (0, 1):
        gb.bfs_set_options(canonical_parents=canonical)
        for r in roots:
            dist, par = gb.sssp(g, int(r), 0.1)
            gb.gb_device_status()
            r = int(r)
            assert float(dist[r]) == 0.0 and int(par[r]) == r
            reached = torch.isfinite(dist)
            assert bool(((par == -1) == ~reached).all())
            du, dv = dist[rows.long()], dist[col.long()]
            assert bool((reached[rows.long()] == reached[col.long()]).all()), "edge leaves the reached set"
            m = reached[rows.long()]
            assert bool((dv[m] <= du[m] + wt[m]).all()), "an edge still relaxes"
            v = torch.nonzero(reached).flatten()
            v = v[v != r]
            p = par[v].long()
            pk = v * n + p
            pos = torch.searchsorted(key, pk).clamp(max=key.numel() - 1)
            assert bool((key[pos] == pk).all()), "parent is not a neighbour"
            assert bool((dist[p] + wt[pos] == dist[v]).all()), "tree edge not tight"
            if canonical:  # no smaller-id neighbour is tight
                first = torch.full((n,), n, dtype=torch.int64, device="cuda")
                cand = (dist[rows.long()] + wt == dist[col.long()]) & reached[col.long()]
                first.scatter_reduce_(0, col.long()[cand], rows.long()[cand], reduce="amin")
                assert torch.equal(first[v], p)
                del first, cand
    gb.bfs_set_options(canonical_parents=0)
    g.free()
