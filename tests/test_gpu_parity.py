"""GPU parity: the CUDA path against the oracle, element by element.

Integer results, so the bar is bit-exactness: edge lists, CSR offsets and
columns, level arrays, and parents in canonical mode (the smallest-id
neighbour one level up, which is unique).  In fast mode any valid parent is
allowed, so parents are checked with the Graph500 validator instead.
Every call goes through the C ABI (paper_2012_13548_gb300.binding).
"""
import itertools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2012_13548_gb300 as gb  # noqa: E402
from paper_2012_13548_gb300 import workloads as W  # noqa: E402
from tests.conftest import oracle_bfs, oracle_graph, roots_for  # noqa: E402
from tests.golden import load_hand_graphs  # noqa: E402

pytestmark = pytest.mark.gpu

DEFAULTS = dict(canonical_parents=0, alpha=14.0, beta=24.0, big_degree=256, ms_alpha=16.0,
                ms_beta=32.0, timeout_ms=5000.0, blocks_per_sm=2)


@pytest.fixture(autouse=True)
def _reset_options():
    gb.bfs_set_options(**DEFAULTS)
    yield
    gb.bfs_set_options(**DEFAULTS)
    gb.gb_device_status()   # no kernel may have recorded an error


def np_(t):
    return t.cpu().numpy()


_graphs = {}


def gpu_graph(scale, index=-1):
    key = (scale, index)
    if key not in _graphs:
        spec = W.GraphSpec(scale=scale, index=index)
        e = gb.kron_generate(**spec.kron_args())
        _graphs[key] = (e, gb.graph_build_csr(e, scale))
    return _graphs[key]


# ---------------------------------------------------------------------------
# Generator (Sec. 2.1) and kernel 1 (Sec. 2.2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("scale", list(range(1, 13)) + [16, 20])
def test_generator_bit_exact(scale):
    e_ref, _, _ = oracle_graph(scale)
    e, _ = gpu_graph(scale)
    assert np.array_equal(np_(e), e_ref)


# the sort's pass plans: 8-bit digits, 9-bit (SCALE 9, 18) and mixed (13, 17)
@pytest.mark.parametrize("scale", list(range(1, 14)) + [16, 17, 18, 20])
def test_csr_bit_exact(scale):
    _, off_ref, col_ref = oracle_graph(scale)
    _, g = gpu_graph(scale)
    off, col = g.csr()
    assert g.n == off_ref.size - 1 and g.nnz == col_ref.size
    assert np.array_equal(np_(off), off_ref)
    assert np.array_equal(np_(col), col_ref)


@pytest.mark.parametrize("scale", [1, 2, 5, 8, 12, 16, 20])
def test_fused_generate_csr_equals_the_two_step_build(scale):
    # generator + kernel 1 without the edge list: the same CSR, bit for bit,
    # as the oracle's build of the oracle's tuples
    spec = W.GraphSpec(scale=scale)
    kw = spec.kron_args()
    G = gb.graph_generate_csr(**kw)
    _, off_ref, col_ref = oracle_graph(scale)
    off, col = G.csr()
    assert np.array_equal(np_(off), off_ref)
    assert np.array_equal(np_(col), col_ref)
    # and the search over it is the search over the two-step graph
    r = roots_for(scale, 1)[0]
    gb.bfs_set_options(canonical_parents=1)
    parent, level = gb.bfs(G, r)
    p_ref, l_ref = oracle_bfs(scale, r)
    assert np.array_equal(np_(level), l_ref) and np.array_equal(np_(parent), p_ref)
    G.free()


def test_fused_generate_csr_other_initiators_and_bad_arguments():
    for (a, b, c, ef) in [(0.25, 0.25, 0.25, 4), (0.45, 0.15, 0.15, 8), (1.0, 0.0, 0.0, 2)]:
        kw = dict(scale=9, edgefactor=ef, a=a, b=b, c=c, seed_gen=11, seed_perm=12, seed_shuf=13)
        G = gb.graph_generate_csr(**kw)
        off_ref, col_ref = oracle.csr_build(oracle.kron_generate(**kw), 9)
        off, col = G.csr()
        assert np.array_equal(np_(off), off_ref) and np.array_equal(np_(col), col_ref), (a, b, c, ef)
        G.free()
    with pytest.raises(gb.GbError, match="INVALID"):
        gb.graph_generate_csr(0, 16, 0.57, 0.19, 0.19, 1, 2)
    with pytest.raises(gb.GbError, match="INVALID"):
        gb.graph_generate_csr(10, 16, 0.6, 0.3, 0.3, 1, 2)


def test_generator_other_initiators_and_edgefactors():
    for (a, b, c, ef, scale) in [(0.25, 0.25, 0.25, 1, 9), (0.45, 0.15, 0.15, 3, 11),
                                 (1.0, 0.0, 0.0, 2, 5), (0.0, 0.0, 0.0, 2, 5)]:
        e = gb.kron_generate(scale, ef, a, b, c, 11, 12, 13)
        ref = oracle.kron_generate(scale, ef, a, b, c, 11, 12, 13)
        assert np.array_equal(np_(e), ref), (a, b, c, ef, scale)


def test_csr_of_hand_fixtures_and_random_lists():
    for g in load_hand_graphs():
        if "off" not in g:
            continue
        scale = max(1, (g["n"] - 1).bit_length())
        e = torch.as_tensor(g["edges"]).cuda()
        G = gb.graph_build_csr(e, scale)
        off, col = G.csr()
        assert np.array_equal(np_(off)[: g["n"] + 1], g["off"])
        assert np.array_equal(np_(col), g["col"])
    rng = np.random.default_rng(3)
    for scale in [1, 2, 3, 5, 8, 11]:
        n = 1 << scale
        for m in [0, 1, 7, 4097, 3 * n]:
            e = rng.integers(0, n, size=(2, m)).astype(np.int64)
            off_ref, col_ref = oracle.csr_build(e, scale)
            G = gb.graph_build_csr(torch.as_tensor(e).cuda(), scale)
            off, col = G.csr()
            assert np.array_equal(np_(off), off_ref), (scale, m)
            assert np.array_equal(np_(col), col_ref), (scale, m)


def test_csr_rejects_out_of_range_endpoints():
    e = torch.tensor([[0, 1, 2], [1, 2, 9]], dtype=torch.int64, device="cuda")
    with pytest.raises(gb.GbError, match="RANGE"):
        gb.graph_build_csr(e, 3)
    e = torch.tensor([[0, -1], [1, 2]], dtype=torch.int64, device="cuda")
    with pytest.raises(gb.GbError, match="RANGE"):
        gb.graph_build_csr(e, 3)


@pytest.mark.parametrize("scale", [1, 2, 5, 8, 12, 16, 20])
def test_counting_sort_build_equals_the_oracle_csr(scale):
    # kernel 1 by counting sort: the same CSR as the oracle's, bit for bit
    e, _ = gpu_graph(scale)
    G = gb.graph_build_csr_counting(e, scale)
    _, off_ref, col_ref = oracle_graph(scale)
    off, col = G.csr()
    assert np.array_equal(np_(off), off_ref)
    assert np.array_equal(np_(col), col_ref)
    r = roots_for(scale, 1)[0]
    _, level = gb.bfs(G, r)
    assert np.array_equal(np_(level), oracle_bfs(scale, r)[1])
    G.free()


def test_counting_sort_build_row_classes_fixtures_and_errors():
    for g in load_hand_graphs():
        if "off" not in g:
            continue
        scale = max(1, (g["n"] - 1).bit_length())
        G = gb.graph_build_csr_counting(torch.as_tensor(g["edges"]).cuda(), scale)
        off, col = G.csr()
        assert np.array_equal(np_(off)[: g["n"] + 1], g["off"]), g["name"]
        assert np.array_equal(np_(col), g["col"]), g["name"]
        G.free()
    rng = np.random.default_rng(17)
    # rows of every sort class: a hub of 8000 neighbours with repeats (the
    # radix-sorted long rows), rows of 33..4096 (block sorts), short rows
    scale = 13
    n = 1 << scale
    hub = np.stack([np.zeros(12000, dtype=np.int64), rng.integers(1, n, 12000)])
    mid = np.stack([np.repeat(np.arange(1, 41), 200), rng.integers(0, n, 40 * 200)])
    rnd = rng.integers(0, n, size=(2, 3 * n))
    loops = np.stack([np.arange(50), np.arange(50)])
    e = np.concatenate([hub, mid, rnd, loops, hub[:, :500]], axis=1).astype(np.int64)
    e = e[:, rng.permutation(e.shape[1])].copy()
    off_ref, col_ref = oracle.csr_build(e, scale)
    assert np.diff(off_ref).max() > 4096
    G = gb.graph_build_csr_counting(torch.as_tensor(e).cuda(), scale)
    off, col = G.csr()
    assert np.array_equal(np_(off), off_ref) and np.array_equal(np_(col), col_ref)
    G.free()
    for scale, m in [(1, 20000), (3, 4097)]:  # two rows of ~10^4 entries; rows of ~10^3
        e = rng.integers(0, 1 << scale, size=(2, m)).astype(np.int64)
        off_ref, col_ref = oracle.csr_build(e, scale)
        G = gb.graph_build_csr_counting(torch.as_tensor(e).cuda(), scale)
        off, col = G.csr()
        assert np.array_equal(np_(off), off_ref) and np.array_equal(np_(col), col_ref), (scale, m)
        G.free()
    for scale in [1, 3, 8, 11]:
        n = 1 << scale
        for m in [0, 1, 7, 3 * n]:
            e = rng.integers(0, n, size=(2, m)).astype(np.int64)
            off_ref, col_ref = oracle.csr_build(e, scale)
            G = gb.graph_build_csr_counting(torch.as_tensor(e).cuda(), scale)
            off, col = G.csr()
            assert np.array_equal(np_(off), off_ref), (scale, m)
            assert np.array_equal(np_(col), col_ref), (scale, m)
            G.free()
    for bad in ([[0, 1, 2], [1, 2, 9]], [[0, -1], [1, 2]]):
        with pytest.raises(gb.GbError, match="RANGE"):
            gb.graph_build_csr_counting(torch.tensor(bad, dtype=torch.int64, device="cuda"), 3)


# ---------------------------------------------------------------------------
# Kernel 2 (Sec. 2.3): single-source BFS
# ---------------------------------------------------------------------------

def check_bfs(G, off_ref, col_ref, root, canonical):
    parent, level = gb.bfs(G, root)
    p_ref, l_ref = oracle.bfs(off_ref, col_ref, root)
    lev = np_(level)
    par = np_(parent)
    assert np.array_equal(lev, l_ref), "levels differ (root %d)" % root
    if canonical:
        assert np.array_equal(par, p_ref), "canonical parents differ (root %d)" % root
    else:
        assert oracle.validate(off_ref, col_ref, root, par, lev) == 0, "invalid tree (root %d)" % root


@pytest.mark.parametrize("canonical", [0, 1])
def test_bfs_hand_fixtures(canonical):
    gb.bfs_set_options(canonical_parents=canonical)
    for g in load_hand_graphs():
        off_ref, col_ref = oracle.csr_build(g["edges"], max(1, (g["n"] - 1).bit_length()))
        off_ref = off_ref[: g["n"] + 1]
        G = gb.graph_from_csr(torch.as_tensor(off_ref).cuda(), torch.as_tensor(col_ref).cuda())
        parent, level = gb.bfs(G, g["root"])
        assert np.array_equal(np_(level), g["levels"]), g["name"]
        if canonical:
            assert np.array_equal(np_(parent), g["parents"]), g["name"]
        else:
            assert oracle.validate(off_ref, col_ref, g["root"], np_(parent), np_(level)) == 0


def _random_graph(rng, n, m):
    e = rng.integers(0, n, size=(2, m)).astype(np.int64)
    scale = max(1, (n - 1).bit_length())
    off, col = oracle.csr_build(e, scale)
    return off[: n + 1].copy(), col


@pytest.mark.parametrize("canonical", [0, 1])
def test_bfs_random_small_graphs_all_roots(canonical):
    gb.bfs_set_options(canonical_parents=canonical)
    rng = np.random.default_rng(5)
    for trial in range(12):
        n = int(rng.integers(1, 200))
        off, col = _random_graph(rng, n, int(rng.integers(0, 3 * n)))
        G = gb.graph_from_csr(torch.as_tensor(off).cuda(), torch.as_tensor(col).cuda())
        for root in range(n):
            check_bfs(G, off, col, root, canonical)


SWITCHES = {
    "default": {},
    "top_down_only": dict(alpha=1e-9),
    "bottom_up_early": dict(alpha=1e9, beta=1e9),
    "flip_flop": dict(alpha=1e9, beta=1e-9),
    "tiny_big_degree": dict(big_degree=1),
    "three_blocks_per_sm": dict(blocks_per_sm=3),
    "one_block_per_sm": dict(blocks_per_sm=1),
}


@pytest.mark.parametrize("mode", list(SWITCHES))
@pytest.mark.parametrize("canonical", [0, 1])
@pytest.mark.parametrize("scale", [4, 8, 10, 12])
def test_bfs_kronecker_direction_modes(scale, canonical, mode):
    gb.bfs_set_options(canonical_parents=canonical, **SWITCHES[mode])
    _, off_ref, col_ref = oracle_graph(scale)
    _, G = gpu_graph(scale)
    roots = roots_for(scale, 8)
    if scale <= 8:
        roots = list(range(1 << scale))       # every vertex, isolated ones included
    for r in roots:
        check_bfs(G, off_ref, col_ref, r, canonical)


@pytest.mark.parametrize("scale,k", [(16, 16), (20, 64)])
@pytest.mark.parametrize("canonical", [0, 1])
def test_bfs_large_scales(scale, k, canonical):
    gb.bfs_set_options(canonical_parents=canonical)
    _, off_ref, col_ref = oracle_graph(scale)
    _, G = gpu_graph(scale)
    for r in roots_for(scale, k):
        parent, level = gb.bfs(G, r)
        p_ref, l_ref = oracle_bfs(scale, r)
        assert np.array_equal(np_(level), l_ref), r
        if canonical:
            assert np.array_equal(np_(parent), p_ref), r
        else:
            assert oracle.validate(off_ref, col_ref, r, np_(parent), np_(level)) == 0, r


@pytest.mark.parametrize("mode", ["default", "bottom_up_early", "flip_flop"])
@pytest.mark.parametrize("canonical", [0, 1])
def test_bfs_rows_longer_than_65535(canonical, mode):
    """The bottom-up list walks read a 16-bit degree saturated at 65535 and
    take the exact one from the offsets for a saturated vertex; a wrong degree
    would cut the vertex's chunks at the next top-down level.  Vertex 1 has
    100001 neighbours (the root and 100000 leaves); its hub is the root, so a
    bottom-up first level finds it through the hub and queues it as a big
    vertex, whose chunks the next (top-down, in flip-flop mode) level expands."""
    gb.bfs_set_options(canonical_parents=canonical, **SWITCHES[mode])
    D, F = 100000, 64
    n = 2 + D + F
    leaves = np.arange(2, 2 + D, dtype=np.int64)
    filler = np.arange(2 + D, n, dtype=np.int64)
    e = np.concatenate([np.stack([np.zeros(1, np.int64), np.ones(1, np.int64)]),
                        np.stack([np.ones(D, np.int64), leaves]),
                        np.stack([np.zeros(F, np.int64), filler])], axis=1)
    off, col = oracle.csr_build(e, (n - 1).bit_length())
    off = off[: n + 1].copy()
    assert off[2] - off[1] == D + 1
    G = gb.graph_from_csr(torch.as_tensor(off).cuda(), torch.as_tensor(col).cuda())
    for root in (0, 1, 2, int(filler[0])):
        check_bfs(G, off, col, root, canonical)
    G.free()


def test_bfs_isolated_root_and_bad_root():
    _, off_ref, col_ref = oracle_graph(10)
    _, G = gpu_graph(10)
    iso = int(np.nonzero(np.diff(off_ref) == 0)[0][0])
    parent, level = gb.bfs(G, iso)
    lev = np_(level)
    assert lev[iso] == 0 and (np.delete(lev, iso) == -1).all()
    assert np_(parent)[iso] == iso
    with pytest.raises(gb.GbError, match="RANGE"):
        gb.bfs(G, G.n)
    with pytest.raises(gb.GbError, match="RANGE"):
        gb.bfs(G, -1)


def test_bfs_stats_count_the_search():
    _, G = gpu_graph(12)
    r = roots_for(12, 1)[0]
    _, level = gb.bfs(G, r)
    st = gb.bfs_last_stats()
    lev = np_(level)
    assert st["nlevels"] == lev.max() + 1
    assert st["reached"] == int((lev >= 0).sum())
    assert st["td_levels"] + st["bu_levels"] == st["nlevels"]
    assert 0 < st["edges_examined"] <= 2 * G.nnz


# ---------------------------------------------------------------------------
# Batched kernel 2: multi-source BFS and a batch of graphs
# ---------------------------------------------------------------------------

MS_SWITCHES = {"default": {}, "top_down": dict(ms_alpha=1e-9, ms_beta=1e-9),
               "bottom_up": dict(ms_alpha=1e9, ms_beta=1e9)}


def check_row(off, col, r, par, lev, p_ref, l_ref, canonical, what):
    """Levels bit-exact; parents bit-exact in canonical mode, else a valid tree."""
    assert np.array_equal(lev, l_ref), what
    if canonical:
        assert np.array_equal(par, p_ref), what
    else:
        assert oracle.validate(off, col, r, par, lev) == 0, what


@pytest.mark.parametrize("canonical", [0, 1])
@pytest.mark.parametrize("mode", list(MS_SWITCHES))
@pytest.mark.parametrize("scale,k", [(6, 64), (10, 1), (10, 7), (12, 64), (16, 64)])
def test_msbfs_rows_equal_single_source(scale, k, mode, canonical):
    gb.bfs_set_options(canonical_parents=canonical, **MS_SWITCHES[mode])
    _, off_ref, col_ref = oracle_graph(scale)
    _, G = gpu_graph(scale)
    roots = roots_for(scale, k)
    if scale == 6:
        roots = [int(x) for x in np.arange(64) % (1 << scale)]   # isolated roots included
    P, L = gb.bfs_batch(G, roots)
    for i, r in enumerate(roots):
        p_ref, l_ref = oracle_bfs(scale, r)
        check_row(off_ref, col_ref, r, np_(P[i]), np_(L[i]), p_ref, l_ref, canonical, (i, r))


@pytest.mark.parametrize("canonical", [0, 1])
def test_msbfs_repeated_roots_and_random_graphs(canonical):
    gb.bfs_set_options(canonical_parents=canonical)
    rng = np.random.default_rng(9)
    for trial in range(6):
        n = int(rng.integers(2, 300))
        off, col = _random_graph(rng, n, int(rng.integers(0, 3 * n)))
        G = gb.graph_from_csr(torch.as_tensor(off).cuda(), torch.as_tensor(col).cuda())
        k = int(rng.integers(1, 65))
        roots = [int(x) for x in rng.integers(0, n, size=k)]
        P, L = gb.bfs_batch(G, roots)
        for i, r in enumerate(roots):
            p_ref, l_ref = oracle.bfs(off, col, r)
            check_row(off, col, r, np_(P[i]), np_(L[i]), p_ref, l_ref, canonical, (trial, i, r))


def _three_hub_csr():
    # hubs 0, 1, 2 with 6000 random neighbours each among 20000 leaves (rows
    # longer than the batched kernel's 4096-entry threshold), plus random
    # leaf-leaf edges so that leaves reach the hubs over several levels
    rng = np.random.default_rng(17)
    n = 20003
    e = [np.stack([np.full(6000, h, np.int64), rng.choice(np.arange(3, n), 6000, replace=False)])
         for h in range(3)]
    e.append(rng.integers(3, n, size=(2, 20000)).astype(np.int64))
    off, col = oracle.csr_build(np.concatenate(e, axis=1), (n - 1).bit_length())
    return off[: n + 1].copy(), col


@pytest.mark.parametrize("canonical", [0, 1])
@pytest.mark.parametrize("mode", list(MS_SWITCHES))
def test_msbfs_rows_longer_than_the_huge_threshold(mode, canonical):
    # the first bottom-up level scans rows above 4096 entries one per warp
    # before the groups of 32; the rows must still equal the oracle's
    gb.bfs_set_options(canonical_parents=canonical, **MS_SWITCHES[mode])
    off, col = _three_hub_csr()
    assert (np.diff(off)[:3] > 4096).all()
    G = gb.graph_from_csr(torch.as_tensor(off).cuda(), torch.as_tensor(col).cuda())
    rng = np.random.default_rng(3)
    roots = [0, 1, 2] + [int(x) for x in rng.integers(3, off.size - 1, size=61)]
    P, L = gb.bfs_batch(G, roots)
    for i, r in enumerate(roots):
        p_ref, l_ref = oracle.bfs(off, col, r)
        check_row(off, col, r, np_(P[i]), np_(L[i]), p_ref, l_ref, canonical, (i, r))
    # one graph through the graph-batch path (byte masks, 8 roots)
    P2, L2 = gb.bfs_multi_graph([G], [roots[:8]])
    for b, r in enumerate(roots[:8]):
        p_ref, l_ref = oracle.bfs(off, col, r)
        check_row(off, col, r, np_(P2[0][b]), np_(L2[0][b]), p_ref, l_ref, canonical, (b, r))
    G.free()


@pytest.mark.parametrize("canonical", [0, 1])
@pytest.mark.parametrize("mode", list(MS_SWITCHES))
def test_msbfs_on_the_degree_ordered_copy(mode, canonical):
    # graph_prepare_batched renumbers the vertices by degree for the batched
    # search (automatic from 2^25 vertices); the rows must still equal the
    # oracle's, parents given as original ids and, in canonical mode, still the
    # smallest-id neighbour one level up
    gb.bfs_set_options(canonical_parents=canonical, **MS_SWITCHES[mode])
    cases = [_three_hub_csr(), _path_and_cycle_csr()]
    for scale in (10, 16):
        _, off_ref, col_ref = oracle_graph(scale)
        cases.append((off_ref, col_ref))
    for ci, (off, col) in enumerate(cases):
        G = gb.graph_from_csr(torch.as_tensor(off).cuda(), torch.as_tensor(col).cuda())
        G.prepare_batched()
        G.prepare_batched()   # a second call keeps the copy
        rng = np.random.default_rng(ci)
        roots = [int(x) for x in rng.integers(0, off.size - 1, size=64)]
        P, L = gb.bfs_batch(G, roots)
        for i, r in enumerate(roots):
            p_ref, l_ref = oracle.bfs(off, col, r)
            check_row(off, col, r, np_(P[i]), np_(L[i]), p_ref, l_ref, canonical, (ci, i, r))
        G.free()


def _path_and_cycle_csr():
    # a 200-vertex path and a 150-vertex cycle: searches 100+ levels deep
    e = [(i, i + 1) for i in range(199)] + [(200 + i, 200 + (i + 1) % 150) for i in range(150)]
    e = np.array(e, dtype=np.int64).T.copy()
    off, col = oracle.csr_build(e, 9)
    return off[: 350 + 1].copy(), col


@pytest.mark.parametrize("canonical", [0, 1])
def test_batched_searches_deeper_than_the_level_history(canonical):
    # levels past the batched kernel's mask history take its per-bit path
    gb.bfs_set_options(canonical_parents=canonical)
    off, col = _path_and_cycle_csr()
    G = gb.graph_from_csr(torch.as_tensor(off).cuda(), torch.as_tensor(col).cuda())
    roots = [0, 199, 100, 57, 200, 275, 349, 3]
    P, L = gb.bfs_batch(G, roots)
    for i, r in enumerate(roots):
        p_ref, l_ref = oracle.bfs(off, col, r)
        assert int(l_ref.max()) >= 74
        check_row(off, col, r, np_(P[i]), np_(L[i]), p_ref, l_ref, canonical, (i, r))
    P2, L2 = gb.bfs_multi_graph([G, G], [roots[:4], roots[4:]])
    for gi, rs in enumerate([roots[:4], roots[4:]]):
        for b, r in enumerate(rs):
            p_ref, l_ref = oracle.bfs(off, col, r)
            check_row(off, col, r, np_(P2[gi][b]), np_(L2[gi][b]), p_ref, l_ref, canonical, (gi, b))


@pytest.mark.parametrize("canonical", [0, 1])
@pytest.mark.parametrize("lo,hi,count", [(4, 9, 32), (12, 18, 32)])
def test_multi_graph_batch_equals_standalone(lo, hi, count, canonical):
    gb.bfs_set_options(canonical_parents=canonical)
    specs = W.batch_specs(count, lo, hi)
    graphs, roots = [], []
    for sp in specs:
        _, off_ref, _ = oracle_graph(sp.scale, sp.index)
        _, G = gpu_graph(sp.scale, sp.index)
        graphs.append(G)
        rs = roots_for(sp.scale, 8, sp.index)
        rs = (rs * 8)[:8]
        roots.append(rs)
    P, L = gb.bfs_multi_graph(graphs, roots)
    for gi, sp in enumerate(specs):
        _, off_ref, col_ref = oracle_graph(sp.scale, sp.index)
        for b, r in enumerate(roots[gi]):
            p_ref, l_ref = oracle_bfs(sp.scale, r, sp.index)
            check_row(off_ref, col_ref, r, np_(P[gi][b]), np_(L[gi][b]), p_ref, l_ref, canonical,
                      (gi, b))


def test_bounded_waits_report_timeout_and_the_context_survives():
    # A 100 ns limit makes the grid-barrier waits run out: every block leaves
    # the kernel, the status word says GB_ERR_TIMEOUT, nothing faults or hangs.
    _, G = gpu_graph(16)
    r = roots_for(16, 1)[0]
    gb.bfs_set_options(timeout_ms=1e-4)
    gb.bfs(G, r)
    with pytest.raises(gb.GbError, match="TIMEOUT"):
        gb.gb_device_status()
    gb.bfs_set_options(timeout_ms=5000.0)
    _, off_ref, col_ref = oracle_graph(16)
    check_bfs(G, off_ref, col_ref, r, canonical=0)
