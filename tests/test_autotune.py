"""Host logic of the autotuner: coordinate descent and the table lookup."""
import json

from paper_2012_13548_gb300 import autotune as AT


def test_descent_finds_the_separable_optimum():
    space = {"a": [1, 2, 3, 4], "b": [10, 20, 30]}
    cost = lambda o: (o["a"] - 3) ** 2 + abs(o["b"] - 20) + 1.0   # noqa: E731
    best, t, trace = AT.descend(cost, space, {"a": 1, "b": 10})
    assert best == {"a": 3, "b": 20} and t == 1.0
    assert all(c >= t for _, c in trace)


def test_descent_keeps_start_when_nothing_is_better():
    space = {"a": [1, 2, 3]}
    best, t, _ = AT.descend(lambda o: 5.0, space, {"a": 2})
    assert best == {"a": 2}


def test_table_lookup_takes_the_nearest_scale(tmp_path):
    path = tmp_path / "t.json"
    path.write_text(json.dumps({"plain/20": {"alpha": 8.0, "median_ms": 0.2},
                                "plain/26": {"alpha": 2.0, "median_ms": 5.0},
                                "multigraph": {"ms_alpha": 4.0, "median_ms": 1.0}}))
    assert AT.tuned_options("plain", 21, str(path)) == {"alpha": 8.0}
    assert AT.tuned_options("plain", 25, str(path)) == {"alpha": 2.0}
    assert AT.tuned_options("multigraph", None, str(path)) == {"ms_alpha": 4.0}
    assert AT.tuned_options("batched", 20, str(path)) == {}


def test_table_lookup_strips_both_timing_fields(tmp_path):
    path = tmp_path / "t.json"
    path.write_text(json.dumps({"plain/20": {"alpha": 32.0, "blocks_per_sm": 1, "mean_ms": 0.1},
                                "batched/20": {"ms_alpha": 1.0, "median_ms": 1.9}}))
    assert AT.tuned_options("plain", 20, str(path)) == {"alpha": 32.0, "blocks_per_sm": 1}
    assert AT.tuned_options("batched", 22, str(path)) == {"ms_alpha": 1.0}


def test_committed_table_holds_only_library_options():
    # every entry of the shipped table must be accepted by bfs_set_options
    # (sssp entries: the bucket width, a positive argument of sssp())
    names = {"canonical_parents", "alpha", "beta", "big_degree", "ms_alpha", "ms_beta",
             "timeout_ms", "blocks_per_sm"}
    table = AT.load_table()
    assert table, "tune_table.json is missing"
    for key, ent in table.items():
        opts = AT.tuned_options(key.split("/")[0], int(key.split("/")[1]) if "/" in key else None)
        if key.startswith("sssp/"):
            assert set(opts) == {"delta"} and opts["delta"] > 0, (key, opts)
            continue
        assert set(opts) <= names, (key, opts)
        if "blocks_per_sm" in opts:
            assert opts["blocks_per_sm"] in (1, 2, 3)


def test_sssp_entries_are_looked_up_by_scale(tmp_path):
    path = tmp_path / "t.json"
    path.write_text(json.dumps({"sssp/20": {"delta": 0.125, "mean_ms": 2.5},
                                "sssp/24": {"delta": 0.075, "mean_ms": 35.0},
                                "plain/22": {"alpha": 14.0}}))
    assert AT.tuned_options("sssp", 21, str(path)) == {"delta": 0.125}
    assert AT.tuned_options("sssp", 23, str(path)) == {"delta": 0.075}
    assert "delta" in AT.SSSP_SPACE and all(d > 0 for d in AT.SSSP_SPACE["delta"])
