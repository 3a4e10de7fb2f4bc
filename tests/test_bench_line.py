"""The bench line's layout on CPU: the comparison the metric is about (the headline's
iterations, SL-MG alone, the paper's schedule, their ms per RHS and the speedups) ends the
JSON line, after every other workload, so that a reader of the line's tail sees it."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_comparison_ends_the_line():
    out = {"metric": bench.METRIC, "value": 9.0, "iterations": {"mean": 215.0},
           "mg_only": {"value": 15.2}, "paper_schedule": {"value": 24.7},
           "workload_1152": {"x": 1}, "serving": {"x": 2}, "ood_shapes": {"x": 3}, "workload_2176": {"x": 4}}
    bench._end_with_comparison(out, 15.2, 9.0, 24.7)
    keys = list(json.loads(json.dumps(out)).keys())
    assert tuple(keys[-len(bench.COMPARISON_KEYS):]) == bench.COMPARISON_KEYS
    assert keys.index("workload_2176") < keys.index("iterations")
    assert out["mg_only_ms_per_rhs"] == 15.2 and out["paper_schedule_ms_per_rhs"] == 24.7
    assert out["speedup_vs_mg_only"] == round(15.2 / 9.0, 3)
    assert out["paper_schedule_speedup_vs_mg_only"] == round(15.2 / 24.7, 3)
