"""Host-side fault injection: device allocations that fail.

Every device allocation of the library goes through one wrapper, which
gb_debug_fail_allocations can make fail as if the device were out of memory.
For each entry point, the k-th allocation of one call is made to fail, for
every k until the call no longer allocates that many times: the call must
report GB_ERR_NOMEM (never crash, never record a device error) and leave the
library holding exactly the device blocks it held before (no leak on any
error path).  Then the same call must succeed.  No GPU fault is involved: the
failure is made on the host, before any kernel sees it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2012_13548_gb300 as gb  # noqa: E402
from paper_2012_13548_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

SCALE = 12
MAX_ALLOCS = 80


@pytest.fixture(scope="module")
def graph():
    spec = W.GraphSpec(scale=SCALE)
    edges = gb.kron_generate(**spec.kron_args())
    g = gb.graph_build_csr(edges, SCALE)
    w = gb.kron_weights(edges.shape[1], spec.seed_weight())
    gw = gb.graph_build_csr_weighted(edges, w, SCALE)
    off, _ = g.csr()
    roots = [int(r) for r in W.select_roots(off.cpu().numpy(), 4, spec.seeds()[3])]
    yield spec, edges, w, g, gw, roots
    gb.debug_fail_allocations(0, 0)


def _free(out):
    for x in (out if isinstance(out, (list, tuple)) else [out]):
        if isinstance(x, gb.Graph):
            x.free()


def check_every_allocation_failure(name, call):
    call_ok = call()            # warm-up: per-thread and per-device state exists now
    _free(call_ok)
    torch.cuda.synchronize()
    live0 = gb.debug_live_allocations()
    for k in range(MAX_ALLOCS):
        gb.debug_fail_allocations(k, 1)
        try:
            out = call()
            failed = False
        except gb.GbError as e:
            assert e.status == gb.binding.GB_ERR_NOMEM, (name, k, str(e))
            failed = True
            out = None
        finally:
            gb.debug_fail_allocations(0, 0)
        _free(out)
        torch.cuda.synchronize()
        assert gb.debug_live_allocations() == live0, "%s leaks after failing allocation %d" % (name, k)
        gb.gb_device_status()   # no kernel recorded an error
        if not failed:
            return k            # the call makes k allocations
    raise AssertionError("%s made more than %d allocations" % (name, MAX_ALLOCS))


def test_generator_and_kernel1_report_nomem_without_leaks(graph):
    spec, edges, w, g, gw, roots = graph
    n_alloc = {}
    n_alloc["kron_generate"] = check_every_allocation_failure(
        "kron_generate", lambda: gb.kron_generate(**spec.kron_args()))
    n_alloc["graph_build_csr"] = check_every_allocation_failure(
        "graph_build_csr", lambda: gb.graph_build_csr(edges, SCALE))
    n_alloc["graph_build_csr_counting"] = check_every_allocation_failure(
        "graph_build_csr_counting", lambda: gb.graph_build_csr_counting(edges, SCALE))
    n_alloc["graph_generate_csr"] = check_every_allocation_failure(
        "graph_generate_csr", lambda: gb.graph_generate_csr(**spec.kron_args()))
    n_alloc["graph_build_csr_weighted"] = check_every_allocation_failure(
        "graph_build_csr_weighted", lambda: gb.graph_build_csr_weighted(edges, w, SCALE))
    off, col = g.csr()
    n_alloc["graph_from_csr"] = check_every_allocation_failure(
        "graph_from_csr", lambda: gb.graph_from_csr(off, col))
    # every one of these allocates: the failures above were really injected
    assert all(v > 0 for v in n_alloc.values()), n_alloc


def test_searches_report_nomem_without_leaks(graph):
    spec, edges, w, g, gw, roots = graph
    n = g.n
    par = torch.empty(n, dtype=torch.int32, device="cuda")
    lev = torch.empty(n, dtype=torch.int32, device="cuda")
    P = torch.empty((len(roots), n), dtype=torch.int32, device="cuda")
    L = torch.empty((len(roots), n), dtype=torch.int32, device="cuda")
    dist = torch.empty(n, dtype=torch.float64, device="cuda")
    r = roots[0]
    counts = {
        "bfs": check_every_allocation_failure("bfs", lambda: gb.bfs(g, r, par, lev)),
        "bfs_batch": check_every_allocation_failure("bfs_batch", lambda: gb.bfs_batch(g, roots, P, L)),
        "bfs_multi_graph": check_every_allocation_failure(
            "bfs_multi_graph", lambda: gb.bfs_multi_graph([g, g], [roots[:2], roots[2:]])),
        "bfs_validate": check_every_allocation_failure(
            "bfs_validate", lambda: gb.bfs_validate(g, r, par, lev, edges)),
        "sssp": check_every_allocation_failure("sssp", lambda: gb.sssp(gw, r, 0.1, dist, par)),
        "sssp_validate": check_every_allocation_failure(
            "sssp_validate", lambda: gb.sssp_validate(gw, r, par, dist, edges)),
    }
    assert all(v > 0 for v in counts.values()), counts
    # after all that, the searches are still right
    gb.bfs(g, r, par, lev)
    assert gb.bfs_validate(g, r, par, lev)["code"] == 0


def test_server_creation_reports_nomem_without_leaks(graph):
    spec, edges, w, g, gw, roots = graph
    small = gb.graph_build_csr(gb.kron_generate(**W.GraphSpec(scale=9).kron_args()), 9)

    def create():
        srv = gb.Server([g, small], mem_budget=1 << 34, single_source_min_vertices=1 << 10)
        srv.close()
        return None

    assert check_every_allocation_failure("server_create", create) > 0
    small.free()


def test_batched_layout_reports_nomem_without_leaks(graph):
    spec, edges, w, g, gw, roots = graph
    off, col = g.csr()

    def build_and_prepare():
        G = gb.graph_from_csr(off, col)
        try:
            G.prepare_batched()
        finally:
            G.free()
        return None

    assert check_every_allocation_failure("graph_prepare_batched", build_and_prepare) > 0
    G = gb.graph_from_csr(off, col).prepare_batched()
    P, L = gb.bfs_batch(G, roots)
    assert gb.bfs_validate(G, roots[0], P[0], L[0])["code"] == 0
    G.free()


def test_injection_arguments_are_checked():
    with pytest.raises(gb.GbError, match="INVALID"):
        gb.debug_fail_allocations(-1, 1)
    with pytest.raises(gb.GbError, match="INVALID"):
        gb.debug_fail_allocations(0, -1)
    gb.debug_fail_allocations(0, 0)
    assert gb.debug_live_allocations() >= 0
    assert np.isfinite(gb.debug_live_allocations())
