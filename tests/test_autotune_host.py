"""Host logic of the TF-group autotuner (no GPU): timings are replaced by a
table, so only the choice, the admissible sizes and the cache run."""
import json

import pytest

from paper_2504_13339_gb300 import autotune as AT


class FakePipeline:
    def __init__(self):
        self.n, self.V, self.W, self.H, self.capacity = 1000, 2, 64, 48, 1 << 22
        self.device = "cpu"
        self.tf_group = self.tf_group_bwd = 0
        self.runs = []

    def composite(self, luts):
        self.runs.append(("fwd", self.tf_group))

    def backward_2d(self, dout):
        self.runs.append(("bwd", self.tf_group_bwd))


class Luts:
    def __init__(self, n_tf):
        self.shape = (n_tf, 256, 4)


@pytest.fixture
def fake_timing(monkeypatch, tmp_path):
    monkeypatch.setenv("XDG_CACHE_HOME", str(tmp_path))
    monkeypatch.setattr(AT.torch.cuda, "get_device_name", lambda d=None: "FakeGPU")
    # milliseconds per (pass, group size), looked up by the last run
    table = {("fwd", 1): 3.0, ("fwd", 2): 2.0, ("fwd", 4): 2.5, ("fwd", 8): 9.0,
             ("bwd", 1): 5.0, ("bwd", 2): 4.0, ("bwd", 4): 1.0}
    return table, tmp_path


def test_tune_picks_the_fastest_admissible_groups_and_caches(monkeypatch, fake_timing):
    table, tmp = fake_timing
    p = FakePipeline()
    monkeypatch.setattr(AT, "_time", lambda fn, reps: (fn(), table[p.runs[-1]])[1])
    res = AT.tune(p, Luts(4), dout=object())
    assert (res["fwd"], res["bwd"]) == (2, 4)
    assert (p.tf_group, p.tf_group_bwd) == (2, 4)
    # with 4 tables a group of 8 (half of it empty) is not tried
    assert "fwd8" not in res["times"] and set(res["times"]) >= {"fwd1", "fwd2", "fwd4"}
    cache = json.load(open(tmp / "veg_gb300" / "autotune.json"))
    key = AT.signature(p, 4) + "|bwd"
    assert cache[key]["fwd"] == 2 and cache[key]["bwd"] == 4
    # a second call reads the cache: nothing is timed again
    q = FakePipeline()
    monkeypatch.setattr(AT, "_time", lambda fn, reps: pytest.fail("timed despite the cache"))
    assert AT.tune(q, Luts(4), dout=object())["fwd"] == 2
    assert (q.tf_group, q.tf_group_bwd) == (2, 4)


def test_one_table_tries_only_group_one_and_keeps_the_backward_default(monkeypatch,
                                                                         fake_timing):
    table, _ = fake_timing
    p = FakePipeline()
    monkeypatch.setattr(AT, "_time", lambda fn, reps: (fn(), table[p.runs[-1]])[1])
    res = AT.tune(p, Luts(1), use_cache=False)
    assert res["fwd"] == 1 and set(res["times"]) == {"fwd1"}
    assert res["bwd"] == 4  # not tuned without an upstream gradient
