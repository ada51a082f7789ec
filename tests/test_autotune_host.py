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
        self.tile_batch = self.tile_batch_bwd = 0
        self.runs = []

    def composite(self, luts):
        self.runs.append(("fwd", self.tf_group, self.tile_batch))

    def backward_2d(self, dout):
        self.runs.append(("bwd", self.tf_group_bwd, self.tile_batch_bwd))


class Luts:
    def __init__(self, n_tf):
        self.shape = (n_tf, 256, 4)


@pytest.fixture
def fake_timing(monkeypatch, tmp_path):
    monkeypatch.setenv("XDG_CACHE_HOME", str(tmp_path))
    monkeypatch.setattr(AT.torch.cuda, "get_device_name", lambda d=None: "FakeGPU")
    # milliseconds per (pass, group size, batch), looked up by the last run
    group_ms = {("fwd", 1): 3.0, ("fwd", 2): 2.0, ("fwd", 4): 2.5, ("fwd", 8): 9.0,
                ("bwd", 1): 5.0, ("bwd", 2): 4.0, ("bwd", 4): 1.0}
    batch_ms = {("fwd", 128): 0.3, ("fwd", 256): 0.2, ("fwd", 512): 0.1,
                ("bwd", 128): 0.2, ("bwd", 256): 0.1, ("bwd", 512): 0.4}
    table = {(k, g, b): t + batch_ms[(k, b)] for (k, g), t in group_ms.items()
             for b in AT.BATCHES}
    return table, tmp_path


def test_tune_picks_the_fastest_admissible_groups_and_batches_and_caches(monkeypatch,
                                                                          fake_timing):
    table, tmp = fake_timing
    p = FakePipeline()
    monkeypatch.setattr(AT, "_time", lambda fn, reps: (fn(), table[p.runs[-1]])[1])
    res = AT.tune(p, Luts(4), dout=object())
    assert (res["fwd"], res["fwd_batch"], res["bwd"], res["bwd_batch"]) == (2, 512, 4, 256)
    assert (p.tf_group, p.tile_batch, p.tf_group_bwd, p.tile_batch_bwd) == (2, 512, 4, 256)
    # with 4 tables a group of 8 (half of it empty) is not tried; every batch is
    assert not any(k.startswith("fwd8") for k in res["times"])
    assert {f"fwd{g}x{b}" for g in (1, 2, 4) for b in AT.BATCHES} <= set(res["times"])
    cache = json.load(open(tmp / "veg_gb300" / "autotune.json"))
    key = AT.signature(p, 4) + "|bwd|batch"
    assert (cache[key]["fwd"], cache[key]["fwd_batch"]) == (2, 512)
    assert (cache[key]["bwd"], cache[key]["bwd_batch"]) == (4, 256)
    # a second call reads the cache: nothing is timed again
    q = FakePipeline()
    monkeypatch.setattr(AT, "_time", lambda fn, reps: pytest.fail("timed despite the cache"))
    assert AT.tune(q, Luts(4), dout=object())["fwd"] == 2
    assert (q.tf_group, q.tile_batch, q.tf_group_bwd, q.tile_batch_bwd) == (2, 512, 4, 256)


def test_one_table_tries_only_group_one_and_keeps_the_backward_default(monkeypatch,
                                                                         fake_timing):
    table, _ = fake_timing
    p = FakePipeline()
    monkeypatch.setattr(AT, "_time", lambda fn, reps: (fn(), table[p.runs[-1]])[1])
    res = AT.tune(p, Luts(1), use_cache=False)
    assert res["fwd"] == 1 and set(res["times"]) == {f"fwd1x{b}" for b in AT.BATCHES}
    assert (res["bwd"], res["bwd_batch"]) == (4, 256)  # not tuned without an upstream gradient
