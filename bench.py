#!/usr/bin/env python3
"""Graph500 BFS benchmark on GB300 (kernel 1 + kernel 2 of arXiv 2012.13548, Sec. 2).

Default workload (SCALE 26, edgefactor 16, 64 roots): one step is
  kernel 1 (CSR build from the device-resident Kronecker edge list),
  64 single-source direction-optimising BFS runs (one per root, each timed),
  one 64-root multi-source BFS of the same roots ("batched").
`value` is the Graph500 figure: the harmonic mean over the timed roots of
m_r / t_r, m_r = input tuples whose start vertex the search reached (Sec. 4.3),
t_r = the bfs() call timed with CUDA events on its stream.  L2 is flushed (a
256 MB write) before every timed call.  Beside it, outside the timed region:
the batched-vs-plain comparison on the SCALE 22 graph (64 roots in one launch
against the harmonic mean of 64 single-source runs), and the CPU baseline on
the same SCALE 26 graph: the paper's parallel BFS (Sec. 2.3.2) on all host
cores and the serial oracle BFS, on a graph the CPU builds itself (and which
must equal the GPU's CSR).

Other workloads (--workload): s20 (SCALE 20), s22ms (SCALE 22, plain vs one
64-root launch), batch32 (32 graphs of SCALE 12..18, 8 roots each),
serve6 (serving loop, p50/p99 latency), sssp22 (kernel 3).

`--impl reference` times the paper's parallel BFS (Sec. 2.3.2, OpenMP on all
host cores; for sssp22 the serial oracle's Dijkstra) on a bounded sample of
the same workload and prints the same JSON line with "impl": "reference".
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2012_13548_gb300 import workloads as W  # noqa: E402

METRIC = "BFS GTEPS (harm. mean, 64 roots) plain vs batched; % HBM peak; p50/p99 ms"
SSSP_METRIC = "SSSP GTEPS (kernel 3, harm. mean over 64 roots)"
L2_FLUSH_BYTES = 256 << 20


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="s26",
                   choices=["s20", "s26", "s22ms", "serve6", "batch32", "sssp22"])
    p.add_argument("--untuned", action="store_true", help="library defaults instead of tune_table.json")
    p.add_argument("--duration", type=float, default=3.0, help="serve6: seconds of arrivals")
    p.add_argument("--rate", type=float, default=None, help="serve6: arrivals per second")
    p.add_argument("--roots", type=int, default=64)
    p.add_argument("--canonical", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0,
                   help="CPU baseline: seconds of the paper's parallel BFS to time")
    p.add_argument("--cpu-threads", type=int, default=0, help="CPU baseline threads (0: all)")
    p.add_argument("--no-c4a", action="store_true", help="skip the SCALE 22 batched-vs-plain record")
    return p.parse_args()


def harmonic_mean(x):
    x = [v for v in x]
    return len(x) / sum(1.0 / v for v in x)


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU; replicas, no data-path collective)
# ---------------------------------------------------------------------------

class Dist:
    def __init__(self, want):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            backend = "nccl" if want == "cuda" else "gloo"
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x):
        if not self.pg:
            return x
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def gather(self, xs):
        """Concatenate per-rank float lists on every rank."""
        if not self.pg:
            return list(xs)
        out = [None] * self.world
        self.pg.all_gather_object(out, list(xs))
        return [v for part in out for v in part]

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def shard_roots(all_roots, rank, world, per_rank):
    """Root list of one rank: ranks take disjoint consecutive blocks."""
    return list(all_roots[rank * per_rank:(rank + 1) * per_rank])


# ---------------------------------------------------------------------------
# clocks under load
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, f in rows for i, v in enumerate(f)
                          if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------

def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def cpu_graph(spec, threads):
    """The workload's graph built on the host by the paper's multicore method
    (Sec. 2.1 generator, Sec. 2.2 CSR, a parallel radix sort as Sec. 4.2
    proposes): (off, col, starts, seconds)."""
    import oracle.parallel as P
    t0 = time.perf_counter()
    off, col, starts = P.kron_csr(**spec.kron_args(), threads=threads)
    return off, col, starts, time.perf_counter() - t0


def cpu_baseline(spec, roots, seconds, threads, gpu_graph=None, gpu_level_of=None):
    """The CPU baseline on the same graph as the GPU line.

    The paper's Algorithm "Parallel BFS" (Sec. 2.3.2, OpenMP on `threads`
    host cores) is timed over the workload's roots until `seconds` of search;
    the serial oracle BFS (Sec. 2.3.1) on the first root beside it.  The graph
    is built on the host by the parallel CPU build; when the GPU's graph is
    given, its CSR must equal the CPU's bit for bit, and the levels of the
    first roots (gpu_level_of(root) -> host int32 array) must equal both CPU
    searches' levels."""
    import oracle
    import oracle.parallel as P
    th = threads or P.max_threads()
    off, col, starts, build_s = cpu_graph(spec, th)
    parity = {}
    if gpu_graph is not None:
        goff, gcol = gpu_graph.csr()
        parity["csr_equal"] = bool(np.array_equal(goff.cpu().numpy(), off) and
                                   np.array_equal(gcol.cpu().numpy(), col))
    rates, spent, done, levels = [], 0.0, 0, {}
    for r in roots:
        t0 = time.perf_counter()
        _, lev, _ = P.bfs(off, col, int(r), threads=th)
        dt = time.perf_counter() - t0
        rates.append(P.teps_edges(starts, lev, th) / dt / 1e9)
        spent += dt
        done += 1
        if done <= 2:
            levels[int(r)] = lev
        if spent >= seconds:
            break
    r0 = int(roots[0])
    t0 = time.perf_counter()
    _, lev_serial = oracle.bfs(off, col, r0)
    ds = time.perf_counter() - t0
    serial = P.teps_edges(starts, lev_serial, th) / ds / 1e9
    if gpu_level_of is not None:
        same = [np.array_equal(gpu_level_of(r), lv) for r, lv in levels.items()]
        parity["levels_equal_roots"] = int(sum(same))
        parity["levels_checked_roots"] = len(same)
        parity["serial_oracle_levels_equal"] = bool(np.array_equal(levels[r0], lev_serial))
    model = cpu_model()
    out = {"value": harmonic_mean(rates), "unit": "GTEPS", "cores": th, "kind": "paper-parallel-bfs",
           "cpu_model": model, "nproc": os.cpu_count(),
           "sample": "the paper's level-synchronous parallel BFS (Sec. 2.3.2, OpenMP, %d threads) on "
                     "the SCALE %d graph built on the host (%.1f s), first %d of its %d roots "
                     "(%.1f s of search)" % (th, spec.scale, build_s, done, len(roots), spent),
           "cpu_kernel1_s": build_s,
           "serial_oracle": {"value": serial, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                             "sample": "serial C oracle queue BFS (Sec. 2.3.1, canonical parents "
                                       "included) from the first root of the same graph (%.1f s)" % ds}}
    if parity:
        out["full_size_parity"] = parity
    return out


def oracle_weighted_graph(scale):
    """The oracle's weighted graph of the workload of `scale`: (edges, off, col, wgt)."""
    import oracle
    spec = W.GraphSpec(scale=scale)
    e = oracle.kron_generate(**spec.kron_args())
    w = oracle.kron_weights(e.shape[1], spec.seed_weight())
    off, col, wgt = oracle.csr_build_weighted(e, w, scale)
    return e, off, col, wgt


def oracle_sssp_sample(scale, nroots, seconds, graph=None):
    """Time the serial oracle Dijkstra over the workload's roots until `seconds`
    of search; returns (harmonic-mean GTEPS, roots timed, seconds spent)."""
    import oracle
    e, off, col, wgt = graph if graph is not None else oracle_weighted_graph(scale)
    roots = W.select_roots(off, nroots, W.GraphSpec(scale=scale).seeds()[3])
    rates, spent, done = [], 0.0, 0
    for r in roots:
        t0 = time.perf_counter()
        d, _ = oracle.sssp(off, col, wgt, int(r))
        dt = time.perf_counter() - t0
        lev = np.where(np.isfinite(d), 0, -1).astype(np.int32)
        rates.append(oracle.teps_edges(e, lev) / dt / 1e9)
        spent += dt
        done += 1
        if spent >= seconds:
            break
    return harmonic_mean(rates), done, spent


def run_reference(args, dist):
    """The reference arm: the paper's parallel BFS (Sec. 2.3.2, OpenMP on all
    host cores) on the workload's graph, built on the host; each step searches
    from the next root.  Under torchrun only rank 0 runs it."""
    if dist.rank != 0:
        return
    wl = W.WORKLOADS[args.workload]
    if args.workload == "sssp22":
        return run_reference_sssp(args, wl)
    if "scale" not in wl:
        print(json.dumps({"impl": "reference",
                          "unavailable": "the %s workload has no CPU counterpart" % args.workload}))
        return
    import oracle.parallel as P
    scale = wl["scale"]
    spec = W.GraphSpec(scale=scale)
    th = args.cpu_threads or P.max_threads()
    off, col, starts, build_s = cpu_graph(spec, th)
    roots = W.select_roots(off, args.roots, spec.seeds()[3])
    rates, step_times = [], []
    i = 0
    for s in range(args.warmup + args.steps):
        r = int(roots[i % len(roots)])
        i += 1
        t0 = time.perf_counter()
        _, lev, _ = P.bfs(off, col, r, threads=th)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            rates.append(P.teps_edges(starts, lev, th) / dt / 1e9)
            step_times.append(dt)
    v = harmonic_mean(rates)
    sample = ("the paper's level-synchronous parallel BFS (Sec. 2.3.2, OpenMP, %d threads) on the "
              "SCALE %d graph built on the host (%.1f s, untimed), one root per step, %d timed steps"
              % (th, scale, build_s, args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GTEPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(step_times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": workload_config(args, scale),
            "cpu_baseline": {"value": v, "unit": "GTEPS", "cores": th, "kind": "paper-parallel-bfs",
                             "cpu_model": cpu_model(), "sample": sample},
            "e2e": {"value": v, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_reference_sssp(args, wl):
    """The oracle's Dijkstra as the reference arm of the kernel-3 workload: each
    step searches from the next few roots of the same graph."""
    import oracle
    scale = wl["scale"]
    e, off, col, wgt = oracle_weighted_graph(scale)
    roots = W.select_roots(off, args.roots, W.GraphSpec(scale=scale).seeds()[3])
    per_step = 2
    rates, step_times = [], []
    i = 0
    for s in range(args.warmup + args.steps):
        t_step = 0.0
        for _ in range(per_step):
            r = int(roots[i % len(roots)])
            i += 1
            t0 = time.perf_counter()
            d, _ = oracle.sssp(off, col, wgt, r)
            dt = time.perf_counter() - t0
            t_step += dt
            if s >= args.warmup:
                lev = np.where(np.isfinite(d), 0, -1).astype(np.int32)
                rates.append(oracle.teps_edges(e, lev) / dt / 1e9)
        if s >= args.warmup:
            step_times.append(t_step)
    v = harmonic_mean(rates)
    sample = ("serial C oracle Dijkstra (binary heap) on the SCALE %d weighted graph (oracle-built), "
              "%d roots per step, %d timed steps" % (scale, per_step, args.steps))
    print(json.dumps({
        "impl": "reference", "metric": SSSP_METRIC, "value": v, "unit": "GTEPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(step_times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": sssp_config(args, wl),
        "cpu_baseline": {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def sssp_delta(args, wl):
    """The bucket width of the kernel-3 workload: tune_table.json's for its
    SCALE unless --untuned, else the workload's default."""
    if args.untuned:
        return wl["delta"]
    from paper_2012_13548_gb300 import autotune
    return autotune.tuned_options("sssp", wl["scale"]).get("delta", wl["delta"])


def sssp_config(args, wl):
    scale = wl["scale"]
    return {"workload": "graph500-kernel3-sssp-kronecker-scale%d-ef16-%droots" % (scale, args.roots),
            "scale": scale, "edgefactor": W.EDGEFACTOR,
            "initiator": [W.A, W.B, W.C, round(1 - W.A - W.B - W.C, 2)],
            "weights": "multiples of 2^-24 in (0, 1], SplitMix64 weight row",
            "roots": args.roots, "delta": sssp_delta(args, wl),
            "options": "tune_table.json" if not args.untuned else "workload default",
            "parents": "canonical" if args.canonical else "any-valid",
            "l2": "flushed before every timed call (256 MB write)",
            "step": "%d single-source shortest-path searches" % args.roots}


def workload_config(args, scale):
    return {"workload": "graph500-kronecker-scale%d-ef16-%droots" % (scale, args.roots),
            "scale": scale, "edgefactor": W.EDGEFACTOR, "initiator": [W.A, W.B, W.C,
                                                                     round(1 - W.A - W.B - W.C, 2)],
            "roots": args.roots, "parents": "canonical" if args.canonical else "any-valid",
            "options": "tune_table.json" if not args.untuned else "library defaults",
            "l2": "flushed before every timed call (256 MB write)",
            "step": "kernel1 + %d single-source BFS + one %d-root batched BFS" % (args.roots, args.roots)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def run_ours(args, dist):
    import torch
    import paper_2012_13548_gb300 as gb

    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    stream = torch.cuda.current_stream()
    wl = W.WORKLOADS[args.workload]
    scale = wl["scale"]
    spec = W.GraphSpec(scale=scale)
    tuned = {}
    if not args.untuned:
        from paper_2012_13548_gb300 import autotune
        tuned = dict(autotune.tuned_options("plain", scale), **autotune.tuned_options("batched", scale))
    gb.bfs_set_options(canonical_parents=args.canonical, **tuned)

    edges = gb.kron_generate(**spec.kron_args())            # input: generated, untimed
    g = gb.graph_build_csr(edges, scale)
    # The degree-ordered copy the batched search runs on for graphs of 2^25
    # vertices and more: built once per graph, like the CSR (a kernel-1
    # structure, Sec. 4.3), and timed here on its own.
    layout_ms = None
    if g.n >= 1 << 25:
        la, lb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        la.record(stream)
        g.prepare_batched(stream)
        lb.record(stream)
        lb.synchronize()
        layout_ms = la.elapsed_time(lb)
    off, _ = g.csr()
    all_roots = W.select_roots(off.cpu().numpy(), args.roots * dist.world, spec.seeds()[3])
    roots = shard_roots(all_roots, dist.rank, dist.world, args.roots)
    n = g.n
    parent = torch.empty(n, dtype=torch.int32, device=dev)
    level = torch.empty(n, dtype=torch.int32, device=dev)
    P = torch.empty((len(roots), n), dtype=torch.int32, device=dev)
    L = torch.empty((len(roots), n), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    # TEPS numerators, per-root counters and the Graph500 validation of every
    # root's tree on the device (bookkeeping, outside the timed region)
    m_r, stats, invalid = [], [], []
    for r in roots:
        gb.bfs(g, int(r), parent, level)
        stats.append(gb.bfs_last_stats())
        v = gb.bfs_validate(g, int(r), parent, level, edges)
        m_r.append(v["teps_edges"])
        if v["code"] != 0:
            invalid.append((int(r), v["code"], v["where"]))
    gb.gb_device_status()

    def step(rec):
        ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
        k0, k1 = ev(), ev()
        flush.fill_(1)
        k0.record(stream)
        g2 = gb.graph_build_csr(edges, scale)
        k1.record(stream)
        per = []
        for r in roots:
            flush.fill_(2)
            a, b = ev(), ev()
            a.record(stream)
            gb.bfs(g, int(r), parent, level)
            b.record(stream)
            per.append((a, b))
        flush.fill_(3)
        b0, b1 = ev(), ev()
        b0.record(stream)
        gb.bfs_batch(g, roots, P, L)
        b1.record(stream)
        # the step's kernel-1 graph (equal to g) is freed at once: graph_free
        # waits for the step's work, and at SCALE 26 every graph holds 9 GB
        g2.free()
        rec.append((k0, k1, per, b0, b1))

    for _ in range(args.warmup):
        step([])
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dist.local)
    clocks.start()
    launches0 = gb.gb_kernel_launches()
    t_all0, t_all1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rec = []
    t_all0.record(stream)
    for _ in range(args.steps):
        step(rec)
    t_all1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    launches = gb.gb_kernel_launches() - launches0
    clk = clocks.stop()
    gb.gb_device_status()
    total_ms = t_all0.elapsed_time(t_all1)

    # generator and kernel 1 fused (no edge list) against the generator plus kernel 1,
    # outside the timed region
    def once(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b), out
    gen_ms, fused_ms, counting_ms = [], [], []
    counting_same = True
    off_g, col_g = g.csr()
    for _ in range(2):
        t, e2 = once(lambda: gb.kron_generate(**spec.kron_args()))
        gen_ms.append(t)
        del e2
        t, g3 = once(lambda: gb.graph_generate_csr(**spec.kron_args()))
        fused_ms.append(t)
        g3.free()
        # kernel 1 by counting sort on the same tuples: timed, and its CSR compared
        t, g4 = once(lambda: gb.graph_build_csr_counting(edges, scale))
        counting_ms.append(t)
        off_c, col_c = g4.csr()
        counting_same = counting_same and bool(torch.equal(off_c, off_g) and torch.equal(col_c, col_g))
        del off_c, col_c
        g4.free()
    del off_g, col_g
    torch.cuda.empty_cache()

    # the batched search's rows (from the last timed step) validated too
    batch_invalid = []
    for i, r in enumerate(roots):
        v = gb.bfs_validate(g, int(r), P[i], L[i])
        if v["code"] != 0:
            batch_invalid.append((int(r), v["code"], v["where"]))
    n_invalid = int(dist.max(float(len(invalid) + len(batch_invalid))))

    bfs_ms = [[a.elapsed_time(b) for (a, b) in r[2]] for r in rec]
    k1_ms = [r[0].elapsed_time(r[1]) for r in rec]
    batch_ms = [r[3].elapsed_time(r[4]) for r in rec]
    rates = [m_r[i] / (t[i] * 1e-3) / 1e9 for t in bfs_ms for i in range(len(roots))]
    all_rates = dist.gather(rates)
    hm = harmonic_mean(all_rates)
    value = hm * dist.world          # replicas run their roots concurrently
    ms_per_step = dist.max(total_ms / args.steps)
    flat_ms = [x for t in bfs_ms for x in t]
    lat = dist.gather(flat_ms)
    batched_gteps = sum(m_r) / (statistics.median(batch_ms) * 1e-3) / 1e9

    # roofline of the dominant kernel (the persistent BFS kernel), algorithmic bytes
    peaks = load_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    alg = [4 * s["edges_examined"] + 32 * s["reached"] + 8 * n for s in stats]
    mean_bytes = statistics.mean(alg)
    mean_ms = statistics.mean(flat_ms)
    achieved = mean_bytes / (mean_ms * 1e-3) / 1e9
    traffic, traffic_note = read_traffic(scale, mean_bytes)
    k1_bytes = kernel1_bytes(edges.shape[1], scale, g.nnz, n)

    # end to end through the public API from pinned host memory
    e2e = None if args.no_e2e else run_e2e(args, gb, torch, edges, scale, roots, m_r, dist)

    # batched vs plain on the SCALE 22 graph (64 roots in one launch against
    # 64 single-source searches), outside the timed region
    c4a = None
    if not args.no_c4a and args.workload != "s22ms":
        c4a = batched_vs_plain(args, gb, torch, 22, dist)
        gb.bfs_set_options(canonical_parents=args.canonical, **tuned)

    cpu = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        def gpu_level_of(r):
            gb.bfs(g, int(r), parent, level)
            return level.cpu().numpy()
        cpu = cpu_baseline(spec, all_roots, args.cpu_seconds, args.cpu_threads, g, gpu_level_of)
    if dist.rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": dist.world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int32", "data": "synthetic", "config": workload_config(args, scale),
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic,
                             "traffic_note": traffic_note,
                             "alg_bytes_per_launch": mean_bytes, "mean_launch_ms": mean_ms,
                             "kernel": "bfs_kernel (persistent, one launch per root)",
                             "peak_source": "measured" if peaks else "fallback"},
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
                "batched": {"gteps": batched_gteps, "ms": statistics.median(batch_ms),
                            "vs_plain": batched_gteps / hm, "roots": len(roots), "scale": scale},
                "batched_scale22": c4a,
                "kernel1": {"ms": statistics.median(k1_ms),
                            "gbs": k1_bytes / (statistics.median(k1_ms) * 1e-3) / 1e9,
                            "frac_of_hbm_peak": k1_bytes / (statistics.median(k1_ms) * 1e-3) / 1e9 / peak,
                            "alg_bytes": k1_bytes,
                            "generator_ms": min(gen_ms),
                            "fused_generate_build_ms": min(fused_ms),
                            "counting_sort_ms": min(counting_ms),
                            "counting_sort_same_csr": counting_same,
                            "batched_layout_ms": layout_ms},
                "validation": {"on": "device (bfs_validate, Graph500 rules 1-7)",
                               "trees": 2 * len(roots) * dist.world, "invalid_max_per_rank": n_invalid,
                               "first_failures": (invalid + batch_invalid)[:4]},
                "latency_ms": {"p50": float(np.percentile(lat, 50)),
                               "p99": float(np.percentile(lat, 99))},
                "graph": {"n": n, "nnz": g.nnz, "m": int(edges.shape[1]),
                          "mean_levels": statistics.mean(s["nlevels"] for s in stats),
                          "mean_edges_examined": statistics.mean(s["edges_examined"] for s in stats)}}
        print(json.dumps(line))


def batched_vs_plain(args, gb, torch, scale, dist):
    """Batched multi-source BFS against the plain search on one graph: the
    harmonic mean of 64 single-source searches (each timed, L2 flushed before
    it) and one 64-root launch (median of 5), both on the SCALE `scale` graph
    with the tuned options of that SCALE; every tree and row validated on the
    device.  Untimed by the step clock."""
    from paper_2012_13548_gb300 import autotune
    spec = W.GraphSpec(scale=scale)
    gb.bfs_set_options(canonical_parents=args.canonical,
                       **(dict(autotune.tuned_options("plain", scale),
                               **autotune.tuned_options("batched", scale)) if not args.untuned else {}))
    stream = torch.cuda.current_stream()
    edges = gb.kron_generate(**spec.kron_args())
    g = gb.graph_build_csr(edges, scale)
    off, _ = g.csr()
    all_roots = W.select_roots(off.cpu().numpy(), args.roots * dist.world, spec.seeds()[3])
    roots = shard_roots(all_roots, dist.rank, dist.world, args.roots)
    n = g.n
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    m_r, bad = [], 0
    for r in roots:
        gb.bfs(g, int(r), parent, level)
        v = gb.bfs_validate(g, int(r), parent, level, edges)
        m_r.append(v["teps_edges"])
        bad += v["code"] != 0
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    plain_rates = []
    for rep in range(3):
        per = []
        for r in roots:
            flush.fill_(rep)
            a, b = ev(), ev()
            a.record(stream)
            gb.bfs(g, int(r), parent, level)
            b.record(stream)
            per.append((a, b))
        torch.cuda.synchronize()
        if rep > 0:
            plain_rates += [m_r[i] / (per[i][0].elapsed_time(per[i][1]) * 1e-3) / 1e9
                            for i in range(len(roots))]
    P = torch.empty((len(roots), n), dtype=torch.int32, device="cuda")
    L = torch.empty((len(roots), n), dtype=torch.int32, device="cuda")
    bms = []
    for rep in range(6):
        flush.fill_(rep)
        a, b = ev(), ev()
        a.record(stream)
        gb.bfs_batch(g, roots, P, L)
        b.record(stream)
        b.synchronize()
        if rep > 0:
            bms.append(a.elapsed_time(b))
    for i, r in enumerate(roots):
        bad += gb.bfs_validate(g, int(r), P[i], L[i])["code"] != 0
    gb.gb_device_status()
    plain = harmonic_mean(dist.gather(plain_rates))
    t_b = dist.max(statistics.median(bms))
    batched = sum(dist.gather(m_r)) / (t_b * 1e-3) / 1e9
    g.free()
    del P, L, edges
    torch.cuda.empty_cache()
    return {"scale": scale, "roots": len(roots) * dist.world,
            "plain_gteps": plain * dist.world, "batched_gteps": batched,
            "vs_plain": batched / (plain * dist.world), "batched_ms": t_b,
            "invalid_trees": int(dist.max(float(bad)))}


def kernel1_bytes(m, scale, nnz, n):
    """Algorithmic HBM bytes of kernel 1: read tuples, write 2m keys, histogram
    read, P sort passes (read+write 16 bytes per key), count + write passes
    (read keys twice), write columns and offsets."""
    nk = 2 * m
    passes = (2 * scale + 7) // 8
    return 16 * m + 8 * nk + 8 * nk + passes * 16 * nk + 16 * nk + 4 * nnz + 8 * (n + 1)


def read_traffic(scale, alg_bytes_per_launch):
    """DRAM bytes per bfs_kernel launch from the committed ncu summary of this
    SCALE, if it was taken on the current kernel source: measured at this
    SCALE (bytes_per_launch), or measured at a smaller one as a ratio of DRAM
    to algorithmic bytes (dram_per_alg_bytes) and scaled by this run's
    algorithmic bytes per launch.  Returns (bytes or None, how it was got)."""
    path = os.path.join(ROOT, "profiles", "bfs_kernel_s%d_traffic.txt" % scale)
    if not os.path.exists(path):
        return None, "no DRAM-counter summary for this SCALE"
    kv = {}
    for line in open(path):
        if "=" in line and not line.lstrip().startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_hash") != kernel_source_hash():
        return None, "the DRAM-counter summary was taken on another kernel source"
    if "bytes_per_launch" in kv:
        return int(kv["bytes_per_launch"]), "ncu DRAM bytes per launch at this SCALE"
    ratio = float(kv["dram_per_alg_bytes"])
    return int(ratio * alg_bytes_per_launch), (
        "ncu DRAM bytes / algorithmic bytes = %.2f measured at SCALE %s, times this run's "
        "algorithmic bytes per launch" % (ratio, kv.get("measured_scale", "?")))


def kernel_source_hash(main="bfs.cu"):
    """Hash of a kernel's code (its file, bfs.cu by default, and common.cuh) with
    comments and whitespace removed: a traffic summary stays valid across
    comment edits and is dropped by any change to the code itself."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in (main, "common.cuh"):
        src = open(os.path.join(ROOT, "paper_2012_13548_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def run_e2e(args, gb, torch, edges, scale, roots, m_r, dist):
    """The same metric end to end: per step the edge list goes host->device from
    pinned memory, kernel 1 builds the graph, and every root's BFS result comes
    back device->host into pinned memory.  A root's time is its BFS plus its
    copy back plus 1/k of the upload and the build."""
    stream = torch.cuda.current_stream()
    h_edges = edges.cpu().pin_memory()
    n = 1 << scale
    d_edges = torch.empty_like(edges)
    parent = torch.empty(n, dtype=torch.int32, device=edges.device)
    level = torch.empty(n, dtype=torch.int32, device=edges.device)
    h_par = torch.empty(n, dtype=torch.int32).pin_memory()
    h_lev = torch.empty(n, dtype=torch.int32).pin_memory()
    k = len(roots)
    rates = []
    for s in range(args.warmup + args.steps):
        ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
        a0, a1 = ev(), ev()
        a0.record(stream)
        d_edges.copy_(h_edges, non_blocking=True)
        g = gb.graph_build_csr(d_edges, scale)
        a1.record(stream)
        per = []
        for r in roots:
            b0, b1 = ev(), ev()
            b0.record(stream)
            gb.bfs(g, int(r), parent, level)
            h_par.copy_(parent, non_blocking=True)
            h_lev.copy_(level, non_blocking=True)
            b1.record(stream)
            per.append((b0, b1))
        torch.cuda.synchronize()
        if s >= args.warmup:
            share = a0.elapsed_time(a1) / k
            rates += [m_r[i] / ((per[i][0].elapsed_time(per[i][1]) + share) * 1e-3) / 1e9
                      for i in range(k)]
        g.free()
    all_rates = dist.gather(rates)
    return {"value": harmonic_mean(all_rates) * dist.world, "unit": "GTEPS",
            "h2d_bytes_per_step": int(h_edges.numel() * 8),
            "d2h_bytes_per_step": int(k * 2 * n * 4)}


# ---------------------------------------------------------------------------
# Kernel 3 workload: single-source shortest paths from 64 roots
# ---------------------------------------------------------------------------

def sssp_bytes(st, n):
    """Algorithmic bytes of one search: 16 per edge relaxed (its 8-byte
    (column, weight) pair and the 8-byte distance of its endpoint), 24 per
    expansion (two offsets and the vertex's own distance), 32 per vertex (the
    distance and three stamps initialised, the distance and parent written)."""
    return 16 * st["scanned"] + 24 * st["processed"] + 32 * n


def run_sssp(args, dist):
    import torch
    import paper_2012_13548_gb300 as gb

    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    stream = torch.cuda.current_stream()
    wl = W.WORKLOADS["sssp22"]
    scale, delta = wl["scale"], sssp_delta(args, wl)
    spec = W.GraphSpec(scale=scale)
    gb.bfs_set_options(canonical_parents=args.canonical)
    edges = gb.kron_generate(**spec.kron_args())             # inputs: generated, untimed
    w = gb.kron_weights(edges.shape[1], spec.seed_weight())
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    a, b = ev(), ev()
    a.record(stream)
    g = gb.graph_build_csr_weighted(edges, w, scale)         # kernel 1 with weights
    b.record(stream)
    b.synchronize()
    k1_ms = a.elapsed_time(b)
    off, _ = g.csr()
    all_roots = W.select_roots(off.cpu().numpy(), args.roots * dist.world, spec.seeds()[3])
    roots = shard_roots(all_roots, dist.rank, dist.world, args.roots)
    n = g.n
    dist_t = torch.empty(n, dtype=torch.float64, device=dev)
    par = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    # TEPS numerators, counters and the device validation of every root's tree
    m_r, stats, invalid = [], [], []
    for r in roots:
        gb.sssp(g, int(r), delta, dist_t, par)
        stats.append(gb.sssp_last_stats())
        v = gb.sssp_validate(g, int(r), par, dist_t, edges)
        m_r.append(v["teps_edges"])
        if v["code"] != 0:
            invalid.append((int(r), v["code"], v["where"]))
    gb.gb_device_status()

    def step(rec):
        per = []
        for r in roots:
            flush.fill_(2)
            x, y = ev(), ev()
            x.record(stream)
            gb.sssp(g, int(r), delta, dist_t, par)
            y.record(stream)
            per.append((x, y))
        rec.append(per)

    for _ in range(args.warmup):
        step([])
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dist.local)
    clocks.start()
    launches0 = gb.gb_kernel_launches()
    t0, t1 = ev(), ev()
    rec = []
    t0.record(stream)
    for _ in range(args.steps):
        step(rec)
    t1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    launches = gb.gb_kernel_launches() - launches0
    clk = clocks.stop()
    gb.gb_device_status()
    # the last timed search's tree validated too
    last = gb.sssp_validate(g, int(roots[-1]), par, dist_t)
    if last["code"] != 0:
        invalid.append((int(roots[-1]), last["code"], last["where"]))
    ms = [[x.elapsed_time(y) for (x, y) in per] for per in rec]
    rates = [m_r[i] / (t[i] * 1e-3) / 1e9 for t in ms for i in range(len(roots))]
    hm = harmonic_mean(dist.gather(rates))
    flat = dist.gather([x for t in ms for x in t])
    peaks = load_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    alg = statistics.mean(sssp_bytes(st, n) for st in stats)
    achieved = alg / (statistics.mean(flat) * 1e-3) / 1e9
    e2e = None if args.no_e2e else run_sssp_e2e(args, gb, torch, edges, w, scale, delta, roots, m_r, dist)
    cpu = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        cs = 20   # the serial oracle builds larger weighted graphs too slowly
        v, done, spent = oracle_sssp_sample(cs, len(all_roots), args.cpu_seconds)
        cpu = {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle",
               "sample": "serial C oracle Dijkstra (binary heap) on the SCALE %d weighted graph of "
                         "the same recipe, rebuilt by the oracle, first %d of its %d roots (%.1f s)"
                         % (cs, done, len(all_roots), spent)}
    if dist.rank == 0:
        print(json.dumps({
            "metric": SSSP_METRIC, "value": hm * dist.world, "unit": "GTEPS", "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dist.max(t0.elapsed_time(t1) / args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": sssp_config(args, wl),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": read_sssp_traffic(scale),
                         "kernel": "sssp_kernel (persistent, one launch per root)",
                         "peak_source": "measured" if peaks else "fallback"},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "latency_ms": {"p50": float(np.percentile(flat, 50)), "p99": float(np.percentile(flat, 99))},
            "kernel1_weighted_ms": k1_ms,
            "validation": {"on": "device (sssp_validate, rules 1-7)", "trees": len(roots) + 1,
                           "invalid": invalid[:4], "n_invalid": len(invalid)},
            "search": {"mean_rounds": statistics.mean(st["rounds"] for st in stats),
                       "mean_buckets": statistics.mean(st["buckets"] for st in stats),
                       "mean_scanned": statistics.mean(st["scanned"] for st in stats),
                       "mean_processed": statistics.mean(st["processed"] for st in stats),
                       "mean_phase_ms": [statistics.mean(st["phase_ns"][k] for st in stats) / 1e6
                                         for k in range(4)]},
            "graph": {"n": n, "nnz": g.nnz, "m": int(edges.shape[1])}}))
    g.free()


def run_sssp_e2e(args, gb, torch, edges, w, scale, delta, roots, m_r, dist):
    """Kernel 3 end to end: per step the tuples and weights go host->device
    from pinned memory, kernel 1 builds the weighted graph, and every root's
    distances and parents come back device->host.  A root's time is its search
    plus its copy back plus 1/k of the upload and the build."""
    stream = torch.cuda.current_stream()
    h_edges = edges.cpu().pin_memory()
    h_w = w.cpu().pin_memory()
    n = 1 << scale
    d_edges, d_w = torch.empty_like(edges), torch.empty_like(w)
    dist_t = torch.empty(n, dtype=torch.float64, device=edges.device)
    par = torch.empty(n, dtype=torch.int32, device=edges.device)
    h_d = torch.empty(n, dtype=torch.float64).pin_memory()
    h_p = torch.empty(n, dtype=torch.int32).pin_memory()
    k = len(roots)
    rates = []
    steps = max(1, min(args.steps, 2))
    for s in range(1 + steps):
        ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
        a0, a1 = ev(), ev()
        a0.record(stream)
        d_edges.copy_(h_edges, non_blocking=True)
        d_w.copy_(h_w, non_blocking=True)
        g = gb.graph_build_csr_weighted(d_edges, d_w, scale)
        a1.record(stream)
        per = []
        for r in roots:
            b0, b1 = ev(), ev()
            b0.record(stream)
            gb.sssp(g, int(r), delta, dist_t, par)
            h_d.copy_(dist_t, non_blocking=True)
            h_p.copy_(par, non_blocking=True)
            b1.record(stream)
            per.append((b0, b1))
        torch.cuda.synchronize()
        if s >= 1:
            share = a0.elapsed_time(a1) / k
            rates += [m_r[i] / ((per[i][0].elapsed_time(per[i][1]) + share) * 1e-3) / 1e9
                      for i in range(k)]
        g.free()
    return {"value": harmonic_mean(dist.gather(rates)) * dist.world, "unit": "GTEPS",
            "h2d_bytes_per_step": int(h_edges.numel() * 8 + h_w.numel() * 4),
            "d2h_bytes_per_step": int(k * n * 12)}


def read_sssp_traffic(scale):
    """DRAM bytes per sssp_kernel launch from the committed ncu summary, if it
    was taken at this SCALE on the current source of the kernel; else None."""
    path = os.path.join(ROOT, "profiles", "sssp_kernel_s%d_traffic.txt" % scale)
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_hash") != kernel_source_hash("sssp.cu"):
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------------------
# Serving workload: resident graphs, open-loop Poisson arrivals
# ---------------------------------------------------------------------------

def run_serve(args, dist):
    import torch
    import paper_2012_13548_gb300 as gb

    torch.cuda.set_device(dist.local)
    wl = W.WORKLOADS["serve6"]
    if not args.untuned:
        from paper_2012_13548_gb300 import autotune
        # the multi-source engine serves the graphs below 2^14 vertices, single-source
        # searches the larger ones: tuned options for each side
        gb.bfs_set_options(**autotune.tuned_options("batched", 20), **autotune.tuned_options("plain", 22))
    rate = args.rate or wl["rate"]
    graphs, edges, offs = [], [], []
    for sc in wl["scales"]:
        spec = W.GraphSpec(scale=sc)
        e = gb.kron_generate(**spec.kron_args())
        g = gb.graph_build_csr(e, sc)
        graphs.append(g)
        edges.append(e)
        offs.append(g.csr()[0].cpu().numpy())
    t, gid, draw = W.poisson_trace(rate, args.duration, len(graphs), seed=W.SEED_ARRIVAL + dist.rank)
    roots = np.empty(t.size, dtype=np.int64)
    for gi in range(len(graphs)):
        sel = gid == gi
        roots[sel] = W.root_from_draw(offs[gi], draw[sel])

    # TEPS numerators: every root of the giant component reaches the same set
    m_of = {}
    reach = []
    for gi, g in enumerate(graphs):
        r0 = int(W.select_roots(offs[gi], 1, W.GraphSpec(scale=wl["scales"][gi]).seeds()[3])[0])
        _, lev = gb.bfs(g, r0)
        reach.append((lev >= 0).cpu().numpy())
        m_of[(gi, -1)] = int((lev[edges[gi][0]] >= 0).sum().item())

    def m_r(gi, r):
        if reach[gi][r]:
            return m_of[(gi, -1)]
        if (gi, r) not in m_of:
            _, lev = gb.bfs(graphs[gi], int(r))
            m_of[(gi, r)] = int((lev[edges[gi][0]] >= 0).sum().item())
        return m_of[(gi, r)]

    total_m = sum(m_r(int(g), int(r)) for g, r in zip(gid, roots))
    budget = 64 << 30

    # warm-up on a short prefix, then the timed trace
    srv = gb.Server(graphs, mem_budget=budget)
    k = min(t.size, 200)
    srv.run_trace(t[:k] - t[0], gid[:k], roots[:k])
    torch.cuda.synchronize()
    clocks = ClockSampler(dist.local)
    clocks.start()
    launches0 = gb.gb_kernel_launches()
    w0 = time.perf_counter()
    lat = srv.run_trace(t, gid, roots)
    wall = time.perf_counter() - w0
    launches = gb.gb_kernel_launches() - launches0
    clk = clocks.stop()
    srv.close()
    gb.gb_device_status()

    # the same stream through the plain per-query path: one bfs() at a time, FIFO
    par = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in graphs]
    lvl = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in graphs]
    for i in range(min(50, t.size)):
        gb.bfs(graphs[int(gid[i])], int(roots[i]), par[int(gid[i])], lvl[int(gid[i])])
    torch.cuda.synchronize()
    plain = np.zeros(t.size)
    p0 = time.perf_counter()
    for i in range(t.size):
        due = p0 + t[i]
        while time.perf_counter() < due:
            pass
        gi = int(gid[i])
        gb.bfs(graphs[gi], int(roots[i]), par[gi], lvl[gi])
        torch.cuda.current_stream().synchronize()
        plain[i] = (time.perf_counter() - due) * 1e3
    plain_wall = time.perf_counter() - p0

    if dist.rank == 0:
        line = {"metric": METRIC, "value": total_m / wall / 1e9, "unit": "GTEPS",
                "n_gpus": dist.world, "steps": 1, "warmup": 1,
                "ms_per_step": wall * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": "serving-6-resident-kronecker-graphs-scale14-24-poisson",
                           "scales": list(wl["scales"]), "rate_per_s": rate,
                           "duration_s": args.duration, "queries": int(t.size),
                           "batch": "queries admitted as slots free up and run concurrently: two "
                                    "single-source searches per graph, each on half the SMs "
                                    "(graphs of 2^14+ vertices; smaller ones: 64 query bits "
                                    "of one multi-source search, admitted per level)",
                           "mem_budget_bytes": budget},
                "serving": {"p50_ms": float(np.percentile(lat, 50)),
                            "p99_ms": float(np.percentile(lat, 99)),
                            "qps": t.size / wall, "gteps": total_m / wall / 1e9,
                            "wall_s": wall},
                "plain_per_query": {"p50_ms": float(np.percentile(plain, 50)),
                                    "p99_ms": float(np.percentile(plain, 99)),
                                    "qps": t.size / plain_wall,
                                    "gteps": total_m / plain_wall / 1e9, "wall_s": plain_wall},
                "gpu_launches": launches, "clocks": clk}
        print(json.dumps(line))


# ---------------------------------------------------------------------------
# Graph batch: 32 Kronecker graphs of SCALE 12..18, 8 roots each, one launch
# ---------------------------------------------------------------------------

def run_batch32(args, dist):
    import torch
    import paper_2012_13548_gb300 as gb
    torch.cuda.set_device(dist.local)
    wl = W.WORKLOADS["batch32"]
    if not args.untuned:
        from paper_2012_13548_gb300 import autotune
        gb.bfs_set_options(**autotune.tuned_options("multigraph"))
    specs = W.batch_specs(wl["graphs"], wl["scale_lo"], wl["scale_hi"])
    graphs, roots, edges = [], [], []
    for sp in specs:
        e = gb.kron_generate(**sp.kron_args())
        g = gb.graph_build_csr(e, sp.scale)
        rs = [int(x) for x in W.select_roots(g.csr()[0].cpu().numpy(), wl["roots"], sp.seeds()[3])]
        graphs.append(g)
        roots.append((rs * wl["roots"])[:wl["roots"]])
        edges.append(e)
    r = wl["roots"]
    P = [torch.empty((r, g.n), dtype=torch.int32, device="cuda") for g in graphs]
    L = [torch.empty((r, g.n), dtype=torch.int32, device="cuda") for g in graphs]
    gb.bfs_multi_graph(graphs, roots, P, L)
    m_tot = sum(int((L[gi][b][edges[gi][0]] >= 0).sum().item())
                for gi in range(len(graphs)) for b in range(r))
    par = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in graphs]
    lev = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in graphs]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def one_launch():
        flush.fill_(1)
        a, b = ev(), ev()
        a.record()
        gb.bfs_multi_graph(graphs, roots, P, L)
        b.record()
        b.synchronize()
        return a.elapsed_time(b)

    def sequential():
        flush.fill_(2)
        a, b = ev(), ev()
        a.record()
        for gi, g in enumerate(graphs):
            for x in roots[gi]:
                gb.bfs(g, x, par[gi], lev[gi])
        b.record()
        b.synchronize()
        return a.elapsed_time(b)

    for _ in range(args.warmup):
        one_launch()
        sequential()
    torch.cuda.synchronize()
    clocks = ClockSampler(dist.local)
    clocks.start()
    launches0 = gb.gb_kernel_launches()
    t_batch = [one_launch() for _ in range(args.steps)]
    launches = gb.gb_kernel_launches() - launches0
    clk = clocks.stop()
    t_seq = [sequential() for _ in range(args.steps)]
    gb.gb_device_status()
    tb, ts = statistics.median(t_batch), statistics.median(t_seq)
    if dist.rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": m_tot / (tb * 1e-3) / 1e9, "unit": "GTEPS",
            "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tb, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": "graph-batch-32-kronecker-scale12-18-8roots",
                       "scales": [sp.scale for sp in specs], "roots_per_graph": r,
                       "l2": "flushed before every timed call (256 MB write)"},
            "batched_one_launch": {"ms": tb, "gteps": m_tot / (tb * 1e-3) / 1e9},
            "sequential_plain": {"ms": ts, "gteps": m_tot / (ts * 1e-3) / 1e9,
                                 "launches": len(graphs) * r},
            "speedup": ts / tb, "gpu_launches": launches, "clocks": clk}))


def main():
    args = parse_args()
    dist = Dist("cpu" if args.impl == "reference" else "cuda")
    try:
        if args.impl == "reference":
            run_reference(args, dist)
        elif args.workload == "serve6":
            run_serve(args, dist)
        elif args.workload == "batch32":
            run_batch32(args, dist)
        elif args.workload == "sssp22":
            run_sssp(args, dist)
        else:
            run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
