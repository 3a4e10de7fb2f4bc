"""Host-side logic of serving and launch-shape tuning, without a GPU: the size buckets'
grid, absorbing layer and V-cycle depth, the network levels the autotuner visits, and
the tuning file's entries reaching the library's table (a host-only table: no device
call is made)."""
import json

import pytest

import __graft_entry__


@pytest.fixture(scope="module")
def helm():
    __graft_entry__.build()
    import paper_2306_17486_gb300 as h
    return h


def test_bucket_config_follows_the_serving_grids():
    from paper_2306_17486_gb300 import serving
    # interior n plus max(16, n/16) absorbing cells per side; coarsest grid at most 72^2
    assert serving.bucket_config(256)[:3] == (288, 16, 4)
    assert serving.bucket_config(512)[:3] == (576, 32, 4)
    assert serving.bucket_config(1024)[:3] == (1152, 64, 5)
    assert serving.bucket_config(2048)[:3] == (2304, 128, 6)
    for n in (96, 160, 320, 640):
        N, abl, levels, maxit = serving.bucket_config(n)
        assert N == n + 2 * max(16, n // 16)
        assert N % (1 << (levels - 1)) == 0 and (N >> (levels - 1)) <= 72
        assert maxit >= 2000


def test_level_heights_halve_down_the_network():
    from paper_2306_17486_gb300.autotune import level_heights
    assert level_heights(576) == [576, 288, 144, 72, 36, 18]
    assert level_heights(288) == [288, 144, 72, 36, 18, 9]
    assert level_heights(100) == [100, 50, 25]   # stops at an odd height


def test_committed_tuning_file_loads_into_the_table(helm, tmp_path):
    from paper_2306_17486_gb300 import autotune
    with open(autotune.DEFAULT_PATH) as f:
        doc = json.load(f)
    helm.tune_clear()
    n_all = sum(len(g["entries"]) for g in doc["grids"])
    assert autotune.apply() == n_all
    for g in doc["grids"]:
        for e in g["entries"]:
            assert helm.tune_get(e["knob"], e["height"], g["batch"]) == e["value"]
    helm.tune_clear()
    # a file naming another grid loads nothing for the grids asked for
    p = tmp_path / "t.json"
    p.write_text(json.dumps({"grids": [{"N": 96, "batch": 2, "entries": [{"knob": "conv_rows", "height": 48,
                                                                          "value": 4}]}]}))
    assert autotune.apply(str(p), grids={(576, 64)}) == 0
    assert autotune.apply(str(p), grids={(96, 2)}) == 1 and helm.tune_get("conv_rows", 48, 2) == 4
    assert helm.tune_get("conv_rows", 48, 3) == 0                                 # other batch: heuristic
    helm.tune_clear()
    assert autotune.apply(str(tmp_path / "missing.json")) == 0
