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
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.read_traffic(20) == 1234
    assert bench.read_traffic(22) is None   # measured on another kernel source
    assert bench.read_traffic(24) is None   # no summary


def test_committed_traffic_summaries_parse():
    for scale in (20, 26):
        path = os.path.join(ROOT, "profiles", "bfs_kernel_s%d_traffic.txt" % scale)
        assert os.path.exists(path), path
        kv = {}
        for line in open(path):
            if "=" in line and not line.lstrip().startswith("#"):
                k, v = line.split("=", 1)
                kv[k.strip()] = v.strip()
        assert int(kv["scale"]) == scale
        assert int(kv["bytes_per_launch"]) > 0
        assert len(kv["source_hash"]) == 16


def test_shard_roots_gives_disjoint_blocks():
    roots = list(range(64))
    parts = [bench.shard_roots(roots, r, 4, 16) for r in range(4)]
    flat = [x for p in parts for x in p]
    assert sorted(flat) == roots and all(len(p) == 16 for p in parts)


def test_harmonic_mean():
    assert bench.harmonic_mean([1.0, 1.0]) == pytest.approx(1.0)
    assert bench.harmonic_mean([1.0, 3.0]) == pytest.approx(1.5)


def test_sssp_traffic_summary_follows_the_kernel_source(tmp_path, monkeypatch):
    path = os.path.join(ROOT, "profiles", "sssp_kernel_s22_traffic.txt")
    assert os.path.exists(path)
    h = bench.kernel_source_hash("sssp.cu")
    assert len(h) == 16 and h != bench.kernel_source_hash()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "sssp_kernel_s22_traffic.txt").write_text(
        "# comment\nscale = 22\ndram_bytes_per_launch = 777\nsource_hash = %s\n" % h)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda main="bfs.cu": h if main == "sssp.cu" else "x")
    assert bench.read_sssp_traffic(22) == 777
    assert bench.read_sssp_traffic(20) is None


def test_sssp_algorithmic_bytes():
    st = {"scanned": 10, "processed": 3}
    assert bench.sssp_bytes(st, 4) == 16 * 10 + 24 * 3 + 32 * 4


def test_sssp_config_is_the_same_for_both_arms():
    import argparse
    from paper_2012_13548_gb300 import autotune
    from paper_2012_13548_gb300 import workloads as W
    wl = W.WORKLOADS["sssp22"]
    tuned = argparse.Namespace(untuned=False, roots=64, canonical=0)
    plain = argparse.Namespace(untuned=True, roots=64, canonical=0)
    assert bench.sssp_delta(tuned, wl) == autotune.tuned_options("sssp", 22).get("delta", wl["delta"])
    assert bench.sssp_delta(plain, wl) == wl["delta"]
    assert bench.sssp_config(tuned, wl)["delta"] == bench.sssp_delta(tuned, wl)


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
