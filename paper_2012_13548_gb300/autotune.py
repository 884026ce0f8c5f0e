"""Autotuner for the BFS launch options, per graph SCALE and call kind.

    python -m paper_2012_13548_gb300.autotune --scales 20 22 26 \
        --out paper_2012_13548_gb300/tune_table.json

For each SCALE it builds the seeded Kronecker graph, then improves the options
by coordinate descent: one option at a time takes each of its candidate values
while the others stay fixed, and the fastest value (CUDA-event time over the
tuning roots, L2 flushed before every timed call: the mean over 16 roots for
single-source searches, whose harmonic-mean rate the slow roots govern; the
median of repeated launches for the batched calls) is kept.  Three call
kinds are tuned:

  plain       bfs(): alpha, beta (direction switch), big_degree (frontier
              vertices split over the grid), blocks_per_sm (resident blocks)
  batched     bfs_batch() with 64 roots: ms_alpha, ms_beta
  multigraph  bfs_multi_graph() over 32 graphs of SCALE 12..18, 8 roots each:
              ms_alpha, ms_beta
  sssp        sssp() on the weighted graph (--sssp): the bucket width delta, an
              argument of the call rather than a library option, scored by
              the mean time over 16 roots

The table maps "plain/<scale>", "batched/<scale>", "sssp/<scale>" and
"multigraph" to option dicts; apply_tuned() loads the entry closest in SCALE.
"""
import argparse
import json
import os
import statistics

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_TABLE = os.path.join(HERE, "tune_table.json")

PLAIN_SPACE = {
    "alpha": [2.0, 4.0, 8.0, 14.0, 32.0, 64.0, 128.0, 256.0, 1024.0],
    "beta": [6.0, 12.0, 24.0, 64.0, 256.0],
    "big_degree": [64, 256, 1024, 4096],
    "blocks_per_sm": [1, 2, 3],
}
MS_SPACE = {
    "ms_alpha": [1.0, 4.0, 16.0, 64.0, 256.0],
    "ms_beta": [2.0, 8.0, 32.0, 128.0],
}
SSSP_SPACE = {
    "delta": [0.03, 0.05, 0.075, 0.1, 0.125, 0.15, 0.2, 0.3],
}


def _timer(torch):
    flush = torch.empty(64 << 20, dtype=torch.int32, device="cuda")

    def timed(fn):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b)
    return timed


def descend(evaluate, space, start, passes=2):
    """Coordinate descent; evaluate(opts) -> milliseconds (lower is better)."""
    best = dict(start)
    best_t = evaluate(best)
    trace = [(dict(best), best_t)]
    for _ in range(passes):
        improved = False
        for key, values in space.items():
            for v in values:
                if v == best.get(key):
                    continue
                cand = dict(best)
                cand[key] = v
                t = evaluate(cand)
                trace.append((cand, t))
                if t < best_t * 0.98:
                    best, best_t, improved = cand, t, True
        if not improved:
            break
    return best, best_t, trace


def tune_scale(scale, roots=8, kinds=("plain", "batched")):
    import torch
    from . import binding as gb
    from . import workloads as W

    spec = W.GraphSpec(scale=scale)
    edges = gb.kron_generate(**spec.kron_args())
    g = gb.graph_build_csr(edges, scale)
    off, _ = g.csr()
    rs = [int(r) for r in W.select_roots(off.cpu().numpy(), roots, spec.seeds()[3])]
    timed = _timer(torch)
    parent = torch.empty(g.n, dtype=torch.int32, device="cuda")
    level = torch.empty(g.n, dtype=torch.int32, device="cuda")
    base = gb.bfs_get_options()
    out = {}

    if "plain" in kinds:
        # the mean time over the roots: a harmonic mean of per-root rates (the
        # reported GTEPS) is governed by the slow roots, which a median hides
        prs = [int(r) for r in W.select_roots(off.cpu().numpy(), max(roots, 16), spec.seeds()[3])]

        def ev_plain(opts):
            gb.bfs_set_options(**opts)
            for r in prs[:2]:
                gb.bfs(g, r, parent, level)          # warm-up
            return statistics.mean(timed(lambda r=r: gb.bfs(g, r, parent, level)) for r in prs)
        start = {k: base[k] for k in PLAIN_SPACE}
        best, t, _ = descend(ev_plain, PLAIN_SPACE, start)
        out["plain/%d" % scale] = dict(best, mean_ms=round(t, 4))
        gb.bfs_set_options(**base)

    if "batched" in kinds:
        k = min(64, len(rs) * 8)
        broots = [int(r) for r in W.select_roots(off.cpu().numpy(), k, spec.seeds()[3])]
        P = torch.empty((len(broots), g.n), dtype=torch.int32, device="cuda")
        L = torch.empty((len(broots), g.n), dtype=torch.int32, device="cuda")

        def ev_batch(opts):
            gb.bfs_set_options(**opts)
            gb.bfs_batch(g, broots, P, L)
            return statistics.median(timed(lambda: gb.bfs_batch(g, broots, P, L)) for _ in range(3))
        start = {k: base[k] for k in MS_SPACE}
        best, t, _ = descend(ev_batch, MS_SPACE, start)
        out["batched/%d" % scale] = dict(best, median_ms=round(t, 4))
        gb.bfs_set_options(**base)
    g.free()
    return out


def tune_sssp(scale, roots=16, start_delta=0.1):
    """The bucket width of sssp() on the weighted graph of `scale`."""
    import torch
    from . import binding as gb
    from . import workloads as W

    spec = W.GraphSpec(scale=scale)
    edges = gb.kron_generate(**spec.kron_args())
    w = gb.kron_weights(edges.shape[1], spec.seed_weight())
    g = gb.graph_build_csr_weighted(edges, w, scale)
    del edges, w
    off, _ = g.csr()
    rs = [int(r) for r in W.select_roots(off.cpu().numpy(), roots, spec.seeds()[3])]
    timed = _timer(torch)
    dist = torch.empty(g.n, dtype=torch.float64, device="cuda")
    parent = torch.empty(g.n, dtype=torch.int32, device="cuda")

    def ev(opts):
        gb.sssp(g, rs[0], opts["delta"], dist, parent)   # warm-up
        return statistics.mean(timed(lambda r=r: gb.sssp(g, r, opts["delta"], dist, parent))
                                for r in rs)
    best, t, _ = descend(ev, SSSP_SPACE, {"delta": start_delta}, passes=1)
    g.free()
    return {"sssp/%d" % scale: dict(best, mean_ms=round(t, 4))}


def tune_multigraph(count=32, lo=12, hi=18, r=8):
    import torch
    from . import binding as gb
    from . import workloads as W

    specs = W.batch_specs(count, lo, hi)
    graphs, roots = [], []
    for sp in specs:
        e = gb.kron_generate(**sp.kron_args())
        gg = gb.graph_build_csr(e, sp.scale)
        graphs.append(gg)
        rs = [int(x) for x in W.select_roots(gg.csr()[0].cpu().numpy(), r, sp.seeds()[3])]
        roots.append((rs * r)[:r])
    P = [torch.empty((r, gg.n), dtype=torch.int32, device="cuda") for gg in graphs]
    L = [torch.empty((r, gg.n), dtype=torch.int32, device="cuda") for gg in graphs]
    timed = _timer(torch)
    base = gb.bfs_get_options()

    def ev(opts):
        gb.bfs_set_options(**opts)
        gb.bfs_multi_graph(graphs, roots, P, L)
        return statistics.median(timed(lambda: gb.bfs_multi_graph(graphs, roots, P, L))
                                 for _ in range(3))
    best, t, _ = descend(ev, MS_SPACE, {k: base[k] for k in MS_SPACE})
    gb.bfs_set_options(**base)
    return {"multigraph": dict(best, median_ms=round(t, 4))}


def load_table(path=DEFAULT_TABLE):
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def tuned_options(kind, scale=None, path=DEFAULT_TABLE):
    """The tuned option dict for `kind` ("plain", "batched", "multigraph",
    "sssp") at the nearest tuned SCALE, or {} if the table has none."""
    table = load_table(path)
    if kind == "multigraph":
        ent = table.get("multigraph", {})
    else:
        keys = [k for k in table if k.startswith(kind + "/")]
        if not keys:
            return {}
        best = min(keys, key=lambda k: abs(int(k.split("/")[1]) - (scale or 0)))
        ent = table[best]
    return {k: v for k, v in ent.items() if k not in ("median_ms", "mean_ms")}


def apply_tuned(kind, scale=None, path=DEFAULT_TABLE):
    """Set the library options to the tuned values for this call kind."""
    from . import binding as gb
    opts = tuned_options(kind, scale, path)
    if opts:
        gb.bfs_set_options(**opts)
    return opts


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--scales", type=int, nargs="+", default=[20, 22])
    p.add_argument("--roots", type=int, default=8)
    p.add_argument("--multigraph", action="store_true")
    p.add_argument("--sssp", action="store_true", help="tune sssp()'s bucket width instead of BFS")
    p.add_argument("--out", default=DEFAULT_TABLE)
    a = p.parse_args()
    table = load_table(a.out)
    for s in a.scales:
        res = tune_sssp(s) if a.sssp else tune_scale(s, a.roots)
        print(json.dumps(res))
        table.update(res)
    if a.multigraph:
        res = tune_multigraph()
        print(json.dumps(res))
        table.update(res)
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    with open(a.out, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    print("wrote", a.out)


if __name__ == "__main__":
    main()
