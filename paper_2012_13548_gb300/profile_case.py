"""Run one small, self-contained case of a library kernel, for profilers.

  python -m paper_2012_13548_gb300.profile_case --kernel bfs --scale 22 --roots 3
  python -m paper_2012_13548_gb300.profile_case --kernel msbfs --scale 20 --roots 64
  python -m paper_2012_13548_gb300.profile_case --kernel k1 --scale 22
  python -m paper_2012_13548_gb300.profile_case --kernel k1counting --scale 26
  python -m paper_2012_13548_gb300.profile_case --kernel sssp --scale 22 --roots 3

It generates the Kronecker graph of the given SCALE on the device, builds the
CSR and then runs the chosen kernel a few times, holding nothing else on the
device (a few GB at SCALE 22), so that a profiler can replay one launch.
"""
import argparse

import torch

from . import binding as gb
from . import workloads as W


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--kernel", choices=["bfs", "msbfs", "k1", "k1counting", "sssp"], default="bfs")
    p.add_argument("--scale", type=int, default=22)
    p.add_argument("--roots", type=int, default=3)
    p.add_argument("--canonical", type=int, default=0)
    p.add_argument("--alpha", type=float, default=None)
    p.add_argument("--beta", type=float, default=None)
    p.add_argument("--blocks-per-sm", type=int, default=None)
    p.add_argument("--delta", type=float, default=0.1, help="sssp: bucket width")
    p.add_argument("--tuned", action="store_true",
                   help="apply tune_table.json's options for this SCALE first (as bench.py does)")
    a = p.parse_args()
    spec = W.GraphSpec(scale=a.scale)
    if a.tuned:
        from . import autotune
        autotune.apply_tuned("plain", a.scale)
        autotune.apply_tuned("batched", a.scale)
    opts = dict(canonical_parents=a.canonical)
    if a.alpha is not None:
        opts["alpha"] = a.alpha
    if a.beta is not None:
        opts["beta"] = a.beta
    if a.blocks_per_sm is not None:
        opts["blocks_per_sm"] = a.blocks_per_sm
    gb.bfs_set_options(**opts)
    edges = gb.kron_generate(**spec.kron_args())
    g = gb.graph_build_csr(edges, a.scale)
    off, _ = g.csr()
    roots = [int(r) for r in W.select_roots(off.cpu().numpy(), max(a.roots, 1), spec.seeds()[3])]
    if a.kernel == "bfs":
        parent = torch.empty(g.n, dtype=torch.int32, device="cuda")
        level = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for r in roots:
            gb.bfs(g, r, parent, level)
            st = gb.bfs_last_stats()
            print("root %d levels %d reached %d edges_examined %d td %d bu %d" % (
                r, st["nlevels"], st["reached"], st["edges_examined"], st["td_levels"],
                st["bu_levels"]))
            print("  per level (us, frontier, step):", [
                ("%.1f" % (t / 1e3), f, d) for t, f, d in
                zip(st["level_ns"], st["level_frontier"], st["level_dir"])])
    elif a.kernel == "msbfs":
        P = torch.empty((len(roots), g.n), dtype=torch.int32, device="cuda")
        L = torch.empty((len(roots), g.n), dtype=torch.int32, device="cuda")
        for _ in range(2):
            gb.bfs_batch(g, roots, P, L)
            print(gb.bfs_last_stats())
    elif a.kernel == "sssp":
        g.free()
        w = gb.kron_weights(edges.shape[1], spec.seed_weight())
        gw = gb.graph_build_csr_weighted(edges, w, a.scale)
        dist = torch.empty(gw.n, dtype=torch.float64, device="cuda")
        parent = torch.empty(gw.n, dtype=torch.int32, device="cuda")
        for r in roots:
            gb.sssp(gw, r, a.delta, dist, parent)
            print("root %d" % r, gb.sssp_last_stats())
        gw.free()
    else:
        g.free()
        build = gb.graph_build_csr if a.kernel == "k1" else gb.graph_build_csr_counting
        for _ in range(2):
            g2 = build(edges, a.scale)
            g2.free()
    gb.gb_device_status()
    torch.cuda.synchronize()
    print("ok")


if __name__ == "__main__":
    main()
