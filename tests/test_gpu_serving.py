"""Serving: continuous batching over resident graphs.

Queries that arrive while others run are admitted into free bit-slots at BFS
level boundaries.  Every served result must equal the same query run alone:
levels bit-exact against bfs() and against the oracle always, parents too in
canonical mode (the smallest-id parent is unique); outside it any valid tree
is allowed, so parents pass the Graph500 validation instead.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2012_13548_gb300 as gb  # noqa: E402
from paper_2012_13548_gb300 import workloads as W  # noqa: E402
from tests.conftest import oracle_graph  # noqa: E402

pytestmark = pytest.mark.gpu

SCALES = (8, 10, 12, 14)


@pytest.fixture(scope="module")
def resident():
    graphs, offs = [], []
    for s in SCALES:
        spec = W.GraphSpec(scale=s)
        e = gb.kron_generate(**spec.kron_args())
        graphs.append(gb.graph_build_csr(e, s))
        offs.append(oracle_graph(s)[1])
    return graphs, offs


def _check_results(srv, graphs, tickets, queries, canonical):
    for t, (gi, r) in zip(tickets, queries):
        par, lev = srv.result(t, gi)
        _, l_alone = gb.bfs(graphs[gi], r)
        assert torch.equal(lev, l_alone), (gi, r)
        _, off, col = oracle_graph(SCALES[gi])
        p_ref, l_ref = oracle.bfs(off, col, r)
        par, lev = par.cpu().numpy(), lev.cpu().numpy()
        assert np.array_equal(lev, l_ref), (gi, r)
        if canonical:
            assert np.array_equal(par, p_ref), (gi, r)
        else:
            assert oracle.validate(off, col, r, par, lev) == 0, (gi, r)
        srv.release(t)


@pytest.mark.parametrize("canonical", [0, 1])
def test_burst_larger_than_the_slots(resident, canonical):
    graphs, offs = resident
    gb.bfs_set_options(canonical_parents=canonical)
    rng = np.random.default_rng(11)
    srv = gb.Server(graphs, mem_budget=1 << 30)
    queries = []
    for _ in range(300):                      # > 64 per graph: slots are reused
        gi = int(rng.integers(0, len(graphs)))
        queries.append((gi, int(rng.integers(0, graphs[gi].n))))   # isolated roots included
    tickets = [srv.submit(gi, r) for gi, r in queries]
    _check_results(srv, graphs, tickets, queries, canonical)
    srv.close()
    gb.bfs_set_options(canonical_parents=0)
    gb.gb_device_status()


def test_admission_by_memory(resident):
    graphs, offs = resident
    # room for the outputs of two queries on the largest graph at a time
    budget = 2 * 8 * graphs[-1].n
    srv = gb.Server(graphs, mem_budget=budget)
    rng = np.random.default_rng(12)
    queries = [(3, int(r)) for r in W.root_from_draw(offs[3], rng.integers(0, 2**62, size=40))]
    tickets = [srv.submit(gi, r) for gi, r in queries]
    _check_results(srv, graphs, tickets, queries, canonical=False)
    srv.close()


@pytest.mark.parametrize("canonical", [0, 1])
def test_poisson_trace_matches_alone_and_replays_identically(resident, canonical):
    graphs, offs = resident
    gb.bfs_set_options(canonical_parents=canonical)
    t, gid, draw = W.poisson_trace(rate=20000.0, duration_s=0.05, n_graphs=len(graphs), seed=5)
    roots = np.array([W.root_from_draw(offs[g], np.array([d], dtype=np.uint64))[0]
                      for g, d in zip(gid, draw)], dtype=np.int64)
    outs = []
    for rep in range(2):
        srv = gb.Server(graphs, mem_budget=1 << 30)
        lat = srv.run_trace(t, gid, roots, keep_results=True)
        assert lat.shape == t.shape and (lat > 0).all()
        levs = []
        for i in range(t.size):
            par, lev = srv.result(i, int(gid[i]))
            levs.append((par.cpu().numpy(), lev.cpu().numpy()))
            srv.release(i)
        srv.close()
        outs.append(levs)
    for i in range(t.size):
        g, r = int(gid[i]), int(roots[i])
        p_alone, l_alone = gb.bfs(graphs[g], r)
        for rep in range(2):
            assert np.array_equal(outs[rep][i][1], l_alone.cpu().numpy()), i
        if canonical:   # the unique tree: identical in both replays and alone
            assert np.array_equal(outs[0][i][0], outs[1][i][0])
            assert np.array_equal(outs[0][i][0], p_alone.cpu().numpy()), i
        else:
            _, off, col = oracle_graph(SCALES[g])
            for rep in range(2):
                assert oracle.validate(off, col, r, outs[rep][i][0], outs[rep][i][1]) == 0, i
    gb.bfs_set_options(canonical_parents=0)


def test_submit_rejects_bad_queries(resident):
    graphs, _ = resident
    srv = gb.Server(graphs, mem_budget=1 << 30)
    with pytest.raises(gb.GbError, match="RANGE"):
        srv.submit(0, graphs[0].n)
    with pytest.raises(gb.GbError, match="RANGE"):
        srv.submit(len(graphs), 0)
    srv.close()


def test_large_graphs_run_one_search_per_query():
    # graphs of 2^14+ vertices are served by concurrent single-source searches;
    # their results follow the canonical_parents option like bfs() itself
    gb.bfs_set_options(canonical_parents=1)
    big = gb.graph_build_csr(gb.kron_generate(**W.GraphSpec(scale=21).kron_args()), 21)
    small = gb.graph_build_csr(gb.kron_generate(**W.GraphSpec(scale=12).kron_args()), 12)
    graphs = [small, big]
    offs = [g.csr()[0].cpu().numpy() for g in graphs]
    rng = np.random.default_rng(21)
    queries = []
    for _ in range(60):
        gi = int(rng.integers(0, 2))
        queries.append((gi, int(W.root_from_draw(offs[gi], rng.integers(0, 2**62, size=1))[0])))
    srv = gb.Server(graphs, mem_budget=3 * 8 * big.n)   # at most three large-graph queries at once
    tickets = [srv.submit(gi, r) for gi, r in queries]
    for t, (gi, r) in zip(tickets, queries):
        par, lev = srv.result(t, gi)
        p_alone, l_alone = gb.bfs(graphs[gi], r)
        assert torch.equal(lev, l_alone), (gi, r)
        assert torch.equal(par, p_alone), (gi, r)
        srv.release(t)
    srv.close()
    gb.bfs_set_options(canonical_parents=0)
    gb.gb_device_status()
