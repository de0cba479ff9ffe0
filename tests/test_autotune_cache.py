"""Host logic of the autotuner's JSON cache (no GPU): the first call times and
stores the winner, later calls apply it without timing, retune times again,
and an unreadable cache file counts as empty. The library-side timing is
replaced by fakes that record what the cache layer asks of them."""
import json

import pytest

from paper_2009_04352_gb300 import autotune


class FakeChannel:
    def __init__(self):
        self.timed = 0
        self.kernel = None

    def autotune(self, steps):
        self.timed += 1
        self.kernel = 4
        return 4, 0.5 + self.timed

    def set_kernel(self, k):
        self.kernel = k


class FakeBatch:
    def __init__(self):
        self.timed = 0
        self.applied = []

    def autotune(self, steps):
        self.timed += 1
        return 8.25

    def config(self):
        return {"form": 2, "streams": 16, "threads": 128, "ctas_per_sm": 5}

    def set_form(self, form, streams):
        self.applied.append(("form", form, streams))

    def set_config(self, threads, ctas):
        self.applied.append(("config", threads, ctas))


@pytest.fixture
def keys(monkeypatch):
    monkeypatch.setattr(autotune, "channel_key", lambda ch: "dev|channel|test")
    monkeypatch.setattr(autotune, "batch_key", lambda b: "dev|batch|test")


def test_channel_cache_roundtrip(tmp_path, keys):
    path = str(tmp_path / "sub" / "autotune.json")
    ch = FakeChannel()
    first = autotune.tune_channel(ch, path, steps=3)
    assert first == {"kernel": 4, "ms_per_step": 1.5, "cached": False} and ch.timed == 1
    again = FakeChannel()
    second = autotune.tune_channel(again, path)
    assert second["cached"] and second["kernel"] == 4 and again.timed == 0 and again.kernel == 4
    third = autotune.tune_channel(again, path, retune=True)
    assert not third["cached"] and again.timed == 1
    with open(path) as fh:
        assert json.load(fh)["dev|channel|test"]["kernel"] == 4


def test_batch_cache_roundtrip(tmp_path, keys):
    path = str(tmp_path / "autotune.json")
    b = FakeBatch()
    first = autotune.tune_batch(b, path)
    assert not first["cached"] and b.timed == 1
    assert first["form"] == 2 and first["streams"] == 16 and first["ms_per_step"] == 8.25
    b2 = FakeBatch()
    second = autotune.tune_batch(b2, path)
    assert second["cached"] and b2.timed == 0
    assert b2.applied == [("form", 2, 16), ("config", 128, 5)]


def test_unreadable_cache_counts_as_empty(tmp_path, keys):
    path = tmp_path / "autotune.json"
    path.write_text("{ not json")
    ch = FakeChannel()
    out = autotune.tune_channel(ch, str(path))
    assert not out["cached"] and ch.timed == 1
    assert json.loads(path.read_text())["dev|channel|test"]["kernel"] == 4
