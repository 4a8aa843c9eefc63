"""The autotuner's file cache: keys, atomic updates, and that a hit applies the cached choice through the
options while a miss runs the autotuner once (a fake system stands in for a handle: nothing runs on a device)."""
import json
import os
import shutil

import pytest

from paper_1602_05716_gb300 import tuning
from paper_1602_05716_gb300.api import OPT_CTAS, OPT_DEEP_WINDOWS, OPT_HELPERS, OPT_PAIRS, OPT_POLICY


@pytest.fixture
def scratch():
    """A scratch directory inside the repository (ignored by git), removed afterwards."""
    d = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", f"tuning_{os.getpid()}")
    os.makedirs(d, exist_ok=True)
    yield d
    shutil.rmtree(d, ignore_errors=True)


class _FakeSystem:
    def __init__(self, choice):
        self.choice = choice
        self.calls = 0
        self.options = {}

    def autotune(self, trial_sweeps):
        self.calls += 1
        return dict(self.choice)

    def set_option(self, opt, value):
        self.options[opt] = value


def test_key_depends_on_device_and_size_mix_only():
    a = tuning.tuning_key([512, 1000, 32768], "GB300", 152)
    assert a == tuning.tuning_key([32768, 1024, 512], "GB300", 152)  # order and nearby sizes share a bucket
    assert a != tuning.tuning_key([512, 1000, 32768], "GB300", 148)
    assert a != tuning.tuning_key([512, 4000, 32768], "GB300", 152)
    assert a != tuning.tuning_key([512, 1000], "GB300", 152)


def test_miss_runs_the_autotuner_then_hits_apply_the_choice(scratch):
    path = os.path.join(scratch, "sub", "tune.json")
    cache = tuning.TuneCache(path)
    s1 = _FakeSystem({"policy": 1, "ctas": 114, "shape": 6, "trial_ms": 15.2})
    choice, hit = tuning.autotune_cached(s1, [600, 900], cache, "GB300", 152)
    assert not hit and s1.calls == 1 and choice["ctas"] == 114
    stored = json.load(open(path))
    assert list(stored.values()) == [{"policy": 1, "ctas": 114, "shape": 6, "trial_ms": 15.2}]
    s2 = _FakeSystem({"policy": 0, "ctas": 152})
    choice2, hit2 = tuning.autotune_cached(s2, [900, 600], tuning.TuneCache(path), "GB300", 152)
    assert hit2 and s2.calls == 0
    # shape 6 = deep windows and helper warps, pairs mode off
    assert s2.options == {OPT_PAIRS: 0, OPT_DEEP_WINDOWS: 1, OPT_HELPERS: 1, OPT_POLICY: 1, OPT_CTAS: 114}
    assert choice2["policy"] == 1
    s3 = _FakeSystem({"policy": 0, "ctas": 76, "trial_ms": 9.0})
    _, hit3 = tuning.autotune_cached(s3, [600, 900], tuning.TuneCache(path), "GB300", 148)
    assert not hit3 and s3.calls == 1 and len(json.load(open(path))) == 2


def test_a_corrupt_cache_is_refused(scratch):
    p = os.path.join(scratch, "t.json")
    with open(p, "w") as f:
        f.write("[1, 2]")
    with pytest.raises(ValueError):
        tuning.TuneCache(p)
