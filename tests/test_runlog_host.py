"""Run records (JSON lines) written by bench.py --log and the studies: each
record keeps the settings that reproduce a run and what it measured."""
import json

import numpy as np

from paper_1006_4247_gb300 import runlog


class _FakeEngine:
    """The attributes and calls engine_summary reads, without a GPU."""
    L = [8, 16]
    NT = [3, 4]
    C = 2
    precision = "fp32"
    seed = 17
    step = 42

    def paths(self):
        return np.array([14, 24], np.int32), np.array([1, 2], np.int32)


def test_records_append_and_read_back(tmp_path):
    f = str(tmp_path / "sub" / "runs.jsonl")
    eng = runlog.engine_summary(_FakeEngine())
    assert eng == {"L": [8, 16], "n_replicas": [3, 4], "copies": 2, "precision": "fp32", "seed": 17,
                   "step": 42, "paths": [14, 24], "ctas_per_replica": [1, 2]}
    r1 = runlog.record(f, "bench", {"workload": "w"}, {"value": 1.5}, engine=eng)
    runlog.record(f, "study_protocol", {"L": 16}, {"t_R": {"plain": 1.0}})
    lines = open(f).read().splitlines()
    assert len(lines) == 2 and json.loads(lines[0]) == r1
    assert [r["kind"] for r in runlog.read(f)] == ["bench", "study_protocol"]
    got = runlog.read(f, kind="bench")
    assert len(got) == 1 and got[0]["results"]["value"] == 1.5 and got[0]["engine"]["seed"] == 17
    assert got[0]["time"].endswith("Z")


def test_autotune_cache_key_names_everything_the_choice_depends_on():
    from paper_1006_4247_gb300 import pt
    k = pt.autotune_cache_key([16, 32], [24, 48], 2, "fp32", 1, 40, "GB300")
    assert k == pt.autotune_cache_key((16, 32), np.array([24, 48]), 2, "fp32", 1, 40, "GB300")
    for other in (pt.autotune_cache_key([16, 32], [24, 48], 2, "fp64", 1, 40, "GB300"),
                  pt.autotune_cache_key([16, 32], [24, 48], 2, "fp32", 1, 20, "GB300"),
                  pt.autotune_cache_key([16, 32], [24, 48], 2, "fp32", 1, 40, "B200"),
                  pt.autotune_cache_key([32, 16], [48, 24], 2, "fp32", 1, 40, "GB300")):
        assert other != k
