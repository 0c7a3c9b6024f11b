"""Host logic of the autotuner cache (paper_2407_06834_gb300/autotune.py):
problem-class keys, recording a tuned result and looking it up, without a
GPU (a stand-in plan supplies info() and autotune())."""
import json

import pytest

from paper_2407_06834_gb300 import autotune


class FakePlan:
    def __init__(self, n_os=64, m=4, L=3, N=262144):
        self._info = {"n_os": n_os, "m": m, "L": L, "N": N}
        self.calls = 0

    def info(self):
        return dict(self._info)

    def autotune(self, stream=None):
        self.calls += 1
        return {"max_items_pts": 128, "unit_points": 512, "team": [0, 0, 2], "ms": 0.9}


@pytest.fixture
def cache(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "autotune.json"
    monkeypatch.setattr(autotune, "CACHE", str(path))
    return path


def test_keys_bucket_n_by_its_logarithm():
    assert autotune.key_of(64, 4, 3, 262144) == "n64_m4_L3_N18"
    assert autotune.key_of(64, 4, 3, 262143) == "n64_m4_L3_N17"
    assert autotune.key_of(128, 6, 9, 4194304) == "n128_m6_L9_N22"
    assert autotune.key_of(64, 4, 3, 1) == autotune.key_of(64, 4, 3, 2)


def test_record_then_lookup(cache):
    assert autotune.lookup(64, 4, 3, 262144) is None
    P = FakePlan()
    res = autotune.tune_and_record(P)
    assert P.calls == 1 and res["unit_points"] == 512
    hit = autotune.lookup(64, 4, 3, 262144)
    assert hit == {"max_items_pts": 128, "unit_points": 512, "team": [0, 0, 2], "ms": 0.9}
    # another class is untouched; the file holds exactly the recorded class
    assert autotune.lookup(128, 6, 9, 4194304) is None
    assert list(json.loads(cache.read_text())) == ["n64_m4_L3_N18"]


def test_classes_accumulate_and_a_broken_file_reads_as_empty(cache):
    autotune.tune_and_record(FakePlan())
    autotune.tune_and_record(FakePlan(n_os=128, m=6, L=9, N=4194304))
    assert sorted(json.loads(cache.read_text())) == ["n128_m6_L9_N22", "n64_m4_L3_N18"]
    cache.write_text("{not json")
    assert autotune.lookup(64, 4, 3, 262144) is None
    autotune.tune_and_record(FakePlan())
    assert autotune.lookup(64, 4, 3, 262144)["team"] == [0, 0, 2]
