"""The allocation-free BFS entry point (bfs_noalloc) against bfs().

bfs_noalloc serves callers that may not allocate device memory: it keeps its
temporaries in a fixed device array inside the library instead of asking the
allocator.  This file is named to be collected last, so that a failure here
cannot hide an earlier test; it passes alone in a fresh process as well as
after the rest of the suite.  Everything goes through the C ABI.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2012_13548_gb300 as gb  # noqa: E402
from paper_2012_13548_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _canonical():
    saved = gb.bfs_get_options()
    gb.bfs_set_options(canonical_parents=1)   # one unique tree: outputs compare exactly
    yield
    gb.bfs_set_options(**saved)


@pytest.mark.parametrize("scale", [12, 20])
def test_noalloc_matches_bfs_on_two_calls_in_a_row(scale):
    spec = W.GraphSpec(scale=scale)
    edges = gb.kron_generate(**spec.kron_args())
    g = gb.graph_build_csr(edges, scale)
    off, col = g.csr()
    roots = [int(r) for r in W.select_roots(off.cpu().numpy(), 2, spec.seeds()[3])]
    n = g.n
    p0 = torch.empty(n, dtype=torch.int32, device="cuda")
    l0 = torch.empty(n, dtype=torch.int32, device="cuda")
    p1 = torch.empty(n, dtype=torch.int32, device="cuda")
    l1 = torch.empty(n, dtype=torch.int32, device="cuda")
    for r in roots:                        # two calls in a row share the scratch
        gb.bfs(g, r, p0, l0)
        gb.bfs_noalloc(off, col, r, p1, l1)
        assert torch.equal(l1, l0), "levels differ from bfs() (root %d)" % r
        assert torch.equal(p1, p0), "parents differ from bfs() (root %d)" % r
    gb.gb_device_status()


def test_noalloc_rejects_graphs_beyond_its_scratch():
    n = (1 << 20) + 1
    off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(0, dtype=torch.int32, device="cuda")
    p = torch.empty(n, dtype=torch.int32, device="cuda")
    l = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(gb.GbError, match="RANGE"):
        gb.bfs_noalloc(off, col, 0, p, l)
    with pytest.raises(gb.GbError, match="RANGE"):
        gb.bfs_noalloc(off[:11], col, 10, p[:10], l[:10])


def _noalloc_vs_bfs_fast_mode(g, off, col, roots):
    """Fast mode (the library default) allows any valid tree: levels must equal
    bfs()'s and the parents must pass the Graph500 validation on the device."""
    n = g.n
    p0 = torch.empty(n, dtype=torch.int32, device="cuda")
    l0 = torch.empty(n, dtype=torch.int32, device="cuda")
    p1 = torch.empty(n, dtype=torch.int32, device="cuda")
    l1 = torch.empty(n, dtype=torch.int32, device="cuda")
    for r in roots:                        # two calls in a row share the scratch
        gb.bfs(g, r, p0, l0)
        gb.bfs_noalloc(off, col, r, p1, l1)
        assert torch.equal(l1, l0), "levels differ from bfs() (root %d)" % r
        v = gb.bfs_validate(g, r, p1, l1)
        assert v["code"] == 0, "bfs_noalloc's tree is not valid: %r (root %d)" % (v, r)
    gb.gb_device_status()


@pytest.mark.parametrize("scale", [12, 20])
def test_noalloc_fast_mode_levels_match_and_trees_are_valid(scale):
    gb.bfs_set_options(canonical_parents=0)
    spec = W.GraphSpec(scale=scale)
    edges = gb.kron_generate(**spec.kron_args())
    g = gb.graph_build_csr(edges, scale)
    off, col = g.csr()
    roots = [int(r) for r in W.select_roots(off.cpu().numpy(), 2, spec.seeds()[3])]
    _noalloc_vs_bfs_fast_mode(g, off, col, roots)
    g.free()


@pytest.mark.parametrize("canonical", [0, 1])
def test_noalloc_on_a_ragged_graph_with_isolated_vertices(canonical):
    # n = 1000 (not a multiple of 32) with vertices 900..999 isolated: the
    # padding bits of the last bitmap word and the empty rows are exercised
    gb.bfs_set_options(canonical_parents=canonical)
    rng = np.random.default_rng(41)
    n = 1000
    u = rng.integers(0, 900, 6000)
    v = rng.integers(0, 900, 6000)
    keep = u != v
    key = np.unique(np.concatenate([u[keep] * n + v[keep], v[keep] * n + u[keep]]))
    rows, cols = key // n, key % n
    off_np = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off_np, rows + 1, 1)
    off_np = np.cumsum(off_np)
    off = torch.as_tensor(off_np).cuda()
    col = torch.as_tensor(cols.astype(np.int32)).cuda()
    g = gb.graph_from_csr(off, col)
    roots = [int(rows[0]), int(rows[len(rows) // 2]), 950]   # 950 is isolated
    if canonical:
        p0 = torch.empty(n, dtype=torch.int32, device="cuda")
        l0 = torch.empty(n, dtype=torch.int32, device="cuda")
        p1 = torch.empty(n, dtype=torch.int32, device="cuda")
        l1 = torch.empty(n, dtype=torch.int32, device="cuda")
        for r in roots:
            gb.bfs(g, r, p0, l0)
            gb.bfs_noalloc(off, col, r, p1, l1)
            assert torch.equal(l1, l0) and torch.equal(p1, p0), r
        gb.gb_device_status()
    else:
        _noalloc_vs_bfs_fast_mode(g, off, col, roots)
    g.free()
