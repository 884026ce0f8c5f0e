"""Host logic of bench.py that decides what the JSON line reports (CPU only)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_summary_is_used_only_for_the_current_kernel_source(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "bfs_kernel_s20_traffic.txt").write_text(
        "# a comment = ignored\nscale = 20\nbytes_per_launch = 1234\nsource_hash = %s\n" % h)
    (prof / "bfs_kernel_s22_traffic.txt").write_text(
        "scale = 22\nbytes_per_launch = 99\nsource_hash = 0000000000000000\n")
    (prof / "bfs_kernel_s26_traffic.txt").write_text(
        "scale = 26\nmeasured_scale = 24\ndram_per_alg_bytes = 2.5\nsource_hash = %s\n" % h)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.read_traffic(20, 1000)[0] == 1234
    assert bench.read_traffic(22, 1000)[0] is None   # measured on another kernel source
    assert bench.read_traffic(24, 1000)[0] is None   # no summary
    b, note = bench.read_traffic(26, 1000)           # a ratio from a smaller SCALE
    assert b == 2500 and "SCALE 24" in note


def test_committed_traffic_summaries_parse():
    for scale in (24, 26):
        path = os.path.join(ROOT, "profiles", "bfs_kernel_s%d_traffic.txt" % scale)
        assert os.path.exists(path), path
        kv = {}
        for line in open(path):
            if "=" in line and not line.lstrip().startswith("#"):
                k, v = line.split("=", 1)
                kv[k.strip()] = v.strip()
        assert int(kv["scale"]) == scale
        assert float(kv["dram_per_alg_bytes"]) > 0
        assert len(kv["source_hash"]) == 16


def test_cpu_baseline_runs_the_papers_parallel_bfs_on_the_same_graph():
    from paper_2012_13548_gb300 import workloads as W
    import oracle.parallel as P
    spec = W.GraphSpec(scale=12)
    off, _, _ = P.kron_csr(**spec.kron_args())
    roots = W.select_roots(off, 8, spec.seeds()[3])
    out = bench.cpu_baseline(spec, roots, seconds=0.05, threads=2)
    assert out["kind"] == "paper-parallel-bfs" and out["cores"] == 2 and out["value"] > 0
    assert "SCALE 12" in out["sample"]
    assert out["serial_oracle"]["cores"] == 1 and out["serial_oracle"]["value"] > 0
    # with a stand-in for the GPU's levels (the oracle's), parity is reported
    import oracle
    out = bench.cpu_baseline(spec, roots, seconds=0.05, threads=2,
                             gpu_level_of=lambda r: oracle.bfs(off, *P.kron_csr(**spec.kron_args())[1:2], r)[1])
    assert out["full_size_parity"]["levels_equal_roots"] == out["full_size_parity"]["levels_checked_roots"]
    assert out["full_size_parity"]["serial_oracle_levels_equal"]
