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


def fixed_bytes(graphs, **options):
    """The device bytes of a server's own state over these graphs."""
    srv = gb.Server(graphs, mem_budget=1 << 40, **options)
    f = srv.stats()["fixed_bytes"]
    srv.close()
    return f


def test_admission_by_memory(resident):
    graphs, offs = resident
    # room for the server's own state and the outputs of two queries on the
    # largest graph at a time
    budget = fixed_bytes(graphs) + 2 * 8 * graphs[-1].n
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
    # at most three large-graph queries at once
    srv = gb.Server(graphs, mem_budget=fixed_bytes(graphs) + 3 * 8 * big.n)
    tickets = [srv.submit(gi, r) for gi, r in queries]
    for t, (gi, r) in zip(tickets, queries):
        par, lev = srv.result(t, gi)
        p_alone, l_alone = gb.bfs(graphs[gi], r)
        assert torch.equal(lev, l_alone), (gi, r)
        assert torch.equal(par, p_alone), (gi, r)
        # and against the oracle: levels and the canonical (smallest-id) tree
        _, off, col = oracle_graph(21 if gi == 1 else 12)
        p_ref, l_ref = oracle.bfs(off, col, r)
        assert np.array_equal(lev.cpu().numpy(), l_ref), (gi, r)
        assert np.array_equal(par.cpu().numpy(), p_ref), (gi, r)
        srv.release(t)
    srv.close()
    gb.bfs_set_options(canonical_parents=0)
    gb.gb_device_status()


def test_budget_must_hold_the_servers_own_state(resident):
    graphs, _ = resident
    f = fixed_bytes(graphs)
    assert f > 0
    with pytest.raises(gb.GbError, match="NOMEM"):
        gb.Server(graphs, mem_budget=f - 1)
    srv = gb.Server(graphs, mem_budget=f)    # holds its state, admits nothing yet
    st = srv.stats()
    assert st["fixed_bytes"] == f and st["used_bytes"] == f and st["budget_bytes"] == f
    srv.close()


@pytest.mark.parametrize("options", [dict(single_source_min_vertices=0),
                                     dict(single_source_min_vertices=1 << 40),
                                     dict(slots_per_graph=1), dict(slots_per_graph=8),
                                     dict(full_grid=1)])
def test_server_options_give_the_same_results(resident, options):
    # every way of serving (single-source slots for every graph, bit slots for
    # every graph, one or eight slots per graph, whole-grid launches) gives
    # each query the result it has alone
    graphs, offs = resident
    gb.bfs_set_options(canonical_parents=1)
    rng = np.random.default_rng(31)
    queries = [(gi, int(W.root_from_draw(offs[gi], rng.integers(0, 2**62, size=1))[0]))
               for gi in rng.integers(0, len(graphs), size=80)]
    srv = gb.Server(graphs, mem_budget=1 << 34, **options)
    tickets = [srv.submit(gi, r) for gi, r in queries]
    _check_results(srv, graphs, tickets, queries, canonical=True)
    srv.close()
    gb.bfs_set_options(canonical_parents=0)
    with pytest.raises(gb.GbError, match="INVALID"):
        gb.Server(graphs, mem_budget=1 << 30, slots_per_graph=9)
    with pytest.raises(KeyError):
        gb.Server(graphs, mem_budget=1 << 30, no_such_option=1)


def test_cancelled_queries_free_their_memory_and_others_complete(resident):
    graphs, offs = resident
    rng = np.random.default_rng(41)
    f = fixed_bytes(graphs)
    # room for every query at once: the client below collects results in
    # ticket order, so a tighter budget could be held by finished queries it
    # has not reached yet
    srv = gb.Server(graphs, mem_budget=1 << 34)
    queries = [(int(gi), int(W.root_from_draw(offs[gi], rng.integers(0, 2**62, size=1))[0]))
               for gi in rng.integers(0, len(graphs), size=120)]
    tickets = [srv.submit(gi, r) for gi, r in queries]
    cancelled = set(tickets[::3])              # queued, running or done: all cancellable
    for t in sorted(cancelled):
        srv.cancel(t)
    with pytest.raises(gb.GbError, match="INVALID"):
        srv.cancel(tickets[0])                  # twice
    keep = [(t, q) for t, q in zip(tickets, queries) if t not in cancelled]
    _check_results(srv, graphs, [t for t, _ in keep], [q for _, q in keep], canonical=False)
    for t in sorted(cancelled):
        with pytest.raises(gb.GbError, match="INVALID"):
            srv.poll(t)
    # every buffer is back: running cancelled queries release theirs as they end
    import time
    t0 = time.time()
    while srv.stats()["used_bytes"] != f and time.time() - t0 < 30:
        time.sleep(0.01)
    st = srv.stats()
    assert st["used_bytes"] == f, st
    assert st["cancelled"] == len(cancelled) and st["released"] == len(keep), st
    srv.close()
    gb.gb_device_status()


def test_a_slow_consumer_holds_its_memory_and_the_rest_waits(resident):
    # a client that keeps its results (does not release them) holds their
    # memory: with room for two queries, the third waits until one is
    # released, then completes; nothing is lost or run twice
    graphs, offs = resident
    f = fixed_bytes(graphs)
    srv = gb.Server(graphs, mem_budget=f + 2 * 8 * graphs[-1].n)
    roots = [int(r) for r in W.root_from_draw(offs[-1], np.arange(3, dtype=np.uint64) * 977 + 5)]
    t = [srv.submit(len(graphs) - 1, r) for r in roots]
    srv.result(t[0], len(graphs) - 1)
    srv.result(t[1], len(graphs) - 1)
    import time
    time.sleep(0.2)
    assert srv.poll(t[2]) is None               # still waiting for memory
    assert srv.stats()["queued"] == 1
    srv.release(t[0])
    par, lev = srv.result(t[2], len(graphs) - 1)
    _, l_alone = gb.bfs(graphs[-1], roots[2])
    assert torch.equal(lev, l_alone)
    srv.release(t[1])
    srv.release(t[2])
    srv.close()


def test_injected_allocation_failures_delay_queries_but_lose_none(resident):
    # output buffers that cannot be allocated now are retried: the queries wait
    # and complete once allocations succeed again
    graphs, offs = resident
    srv = gb.Server(graphs, mem_budget=1 << 34)
    gb.debug_fail_allocations(0, 6)
    queries = [(gi, int(W.root_from_draw(offs[gi], np.array([7 + gi], dtype=np.uint64))[0]))
               for gi in range(len(graphs))]
    tickets = [srv.submit(gi, r) for gi, r in queries]
    import time
    time.sleep(0.2)
    gb.debug_fail_allocations(0, 0)
    _check_results(srv, graphs, tickets, queries, canonical=False)
    srv.close()
