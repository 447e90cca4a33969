"""Tile-autotuner selection logic on the host: fake batches and simulations, fake timings."""
import types

import pytest


class FakeBatch:
    def __init__(self):
        self.tile = None

    def set_tile(self, t, r):
        self.tile = (t, r)

    def step(self, k):
        pass


@pytest.fixture
def autotune(monkeypatch, tmp_path):
    import torch
    from paper_1110_5004_gb300 import autotune as at
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a, **k: None)
    monkeypatch.setattr(at, "CACHE", str(tmp_path / "cache.json"))
    monkeypatch.setattr(at, "_device_name", lambda: "dev")
    return at


def test_batch_tuner_picks_the_fastest_per_step(autotune, monkeypatch):
    """The fastest candidate wins even when it beats the first one by less than a factor two
    (the timed call advances two steps; candidates are compared per step)."""
    times = {(t, r): 10.0 for t in autotune.BATCH_THREADS for r in autotune.BATCH_ROWS}
    first = next(iter(times))
    times[first] = 6.0
    times[(128, 32)] = 4.0
    b = FakeBatch()
    monkeypatch.setattr(autotune, "_time", lambda fn, reps, stream: times[b.tile])
    t, r, ms = autotune.tune_batch(b)
    assert (t, r) == (128, 32) and b.tile == (128, 32)
    assert ms == pytest.approx(2.0)


def test_sim_tuner_caches_per_storage(autotune, monkeypatch):
    """Tiles are cached per population storage: a 16-bit simulation does not reuse the FP32
    entry of the same grid."""
    calls = []

    class FakeSim:
        def __init__(self, storage):
            self.nx, self.ny, self.params = 300, 200, types.SimpleNamespace(storage=storage)
            self.tile = None

        def set_stream(self, s):
            pass

        def set_tile(self, t, r):
            self.tile = (t, r)

        def step(self, n):
            pass

    def fake_time(fn, reps, stream):
        calls.append(1)
        return 1.0 + 0.01 * len(calls)          # the first candidate is the fastest

    monkeypatch.setattr(autotune, "_time", fake_time)
    a = autotune.tune_sim(FakeSim(0))
    n0 = len(calls)
    b = autotune.tune_sim(FakeSim(1))
    assert len(calls) == 2 * n0                  # measured again for the other storage
    c = autotune.tune_sim(FakeSim(1))
    assert len(calls) == 2 * n0 and tuple(c[:2]) == tuple(b[:2])   # then taken from the cache
    assert tuple(a[:2]) == (autotune.THREADS[0], autotune.ROWS[0])
