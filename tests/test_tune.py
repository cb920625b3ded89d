"""Host logic of the launch-shape autotuner (no GPU): candidates per radius, cache
keys, the JSON cache's round trip and its tolerance of damaged files, and the
choice of the fastest shape from measured times."""
import json

import paper_1901_09971_gb300 as dgf
from paper_1901_09971_gb300 import tune


def test_candidates_follow_the_compile_time_layouts():
    assert tune.candidates(4) == (8, 16, 32) and tune.candidates(5) == (8, 16, 32)
    assert tune.candidates(3) == (32,) and tune.candidates(7) == (32,)


def test_key_separates_what_changes_the_work():
    p = dgf.RlofParams(levels=3, radius=4)
    k = tune.key("GB300", p, 3_800_000)
    assert k == "GB300|r4|L3|it30|m4|s0|cross0|pts2^22"
    assert tune.key("GB300", p, 3_000_000) == k  # same size class
    assert tune.key("GB300", p, 900_000) != k
    assert tune.key("GB300", dgf.RlofParams(levels=3, radius=4, storage=dgf.F16), 3_800_000) != k
    assert tune.key("GB300", dgf.RlofParams(levels=3, radius=4, cross_tau=20.0), 3_800_000) != k
    assert tune.key("B200", p, 3_800_000) != k


def test_tune_records_the_fastest_and_lookup_returns_it(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    times = {8: 3.0, 16: 2.5, 32: 4.0}
    seen = []

    def measure(lanes):
        seen.append(lanes)
        return times[lanes]

    rec = tune.tune(measure, 5, "k1", path)
    assert seen == [8, 16, 32] and rec["lanes"] == 16 and rec["ms"] == {"8": 3.0, "16": 2.5, "32": 4.0}
    assert tune.lookup("k1", path) == 16 and tune.lookup("other", path) is None
    tune.tune(lambda lanes: 1.0, 6, "k2", path)  # radius 6: only 32 lanes
    assert tune.lookup("k2", path) == 32 and tune.lookup("k1", path) == 16
    assert tune.choose({8: 1.0, 16: 1.0, 32: 2.0}) == 8


def test_damaged_or_foreign_cache_files_are_ignored(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    assert tune.lookup("k", str(path)) is None
    path.write_text(json.dumps({"version": 999, "entries": {"k": {"lanes": 8}}}))
    assert tune.lookup("k", str(path)) is None
    path.write_text(json.dumps({"version": tune.CACHE_VERSION, "entries": {"k": {"lanes": 12}}}))
    assert tune.lookup("k", str(path)) is None  # not a lane count the library honours
    rec = tune.tune(lambda lanes: {8: 2.0, 16: 1.0, 32: 3.0}[lanes], 4, "k", str(path))
    assert rec["lanes"] == 16 and tune.lookup("k", str(path)) == 16
