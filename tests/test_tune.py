"""The batch-plan tuner's selection and file logic (no GPU): the fastest chunk
length per (n, T-bucket), ties to the longer chunk, the library's entry order,
and a JSON round trip that rejects malformed entries."""
import json

import pytest

from paper_2104_03186_gb300 import tune


def test_choose_picks_fastest_and_breaks_ties_to_longer_chunks():
    timings = {(16, 4096): {32: 5.0, 64: 4.0, 128: 4.0}, (8, 512): {8: 1.0, 16: 2.0},
               (8, 4096): {}}
    entries = tune.choose(timings)
    assert [(e["n"], e["t_max"], e["chunk_steps"]) for e in entries] == [(8, 512, 8),
                                                                        (16, 4096, 128)]
    assert entries[1]["ms"] == {"32": 5.0, "64": 4.0, "128": 4.0}


def test_entries_sorted_for_the_library_and_round_trip(tmp_path):
    plan = {"entries": [{"n": 16, "t_max": 4096, "chunk_steps": 64},
                        {"n": 8, "t_max": 2048, "chunk_steps": 32},
                        {"n": 8, "t_max": 512, "chunk_steps": 16}], "persistent": False}
    path = str(tmp_path / "plan.json")
    tune.save(plan, path)
    back = tune.load(path)
    assert back == plan
    assert tune.entries_for(back) == [(8, 512, 16), (8, 2048, 32), (16, 4096, 64)]


def test_load_rejects_bad_entries(tmp_path):
    path = tmp_path / "bad.json"
    path.write_text(json.dumps({"entries": [{"n": 8, "t_max": 100, "chunk_steps": 0}]}))
    with pytest.raises(ValueError):
        tune.load(str(path))


def test_committed_plan_if_present_is_valid():
    import os

    if not os.path.exists(tune.DEFAULT_OUT):
        pytest.skip("no tuned plan committed")
    plan = tune.load(tune.DEFAULT_OUT)
    assert {e["n"] for e in plan["entries"]} <= {8, 16, 32}
    assert all(e["chunk_steps"] in plan["candidates"] for e in plan["entries"])


def test_choose_mode_prefers_the_small_batch_among_the_near_fastest():
    # auto within 1% of the best on the whole batch and fastest on the small one
    assert tune.choose_mode({"per_level": 45.8, "persistent": 47.3, "auto": 46.1},
                            {"per_level": 0.50, "persistent": 0.42, "auto": 0.42}) == "auto"
    # persistent is fastest on the small batch but too slow on the whole batch
    assert tune.choose_mode({"per_level": 45.8, "persistent": 47.3, "auto": 47.0},
                            {"per_level": 0.50, "persistent": 0.40, "auto": 0.41}) == "per_level"
    # ties go in MODES order
    assert tune.choose_mode({"per_level": 1.0, "persistent": 1.0, "auto": 1.0},
                            {"per_level": 2.0, "persistent": 2.0, "auto": 2.0}) == "per_level"


def test_plan_mode_reads_old_and_new_plans(tmp_path):
    assert tune.plan_mode({"entries": [], "launch_mode": "auto"}) == "auto"
    assert tune.plan_mode({"entries": [], "persistent": False}) == "per_level"
    assert tune.plan_mode({"entries": [], "persistent": True}) == "persistent"
    path = tmp_path / "bad_mode.json"
    path.write_text(json.dumps({"entries": [], "launch_mode": "sometimes"}))
    with pytest.raises(ValueError):
        tune.load(str(path))
