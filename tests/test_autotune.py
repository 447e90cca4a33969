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
    monkeypatch.setattr(at, "_sm_count", lambda: 152)
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


@pytest.mark.parametrize("nx,ny,threads,sms", [(2048, 512, 128, 152), (2048, 512, 256, 152), (4096, 4096, 256, 152),
                                               (128, 128, 128, 152), (300, 77, 64, 10)])
def test_balanced_rows_fill_whole_waves(autotune, nx, ny, threads, sms):
    """Each balanced height is the shortest whose CTA count fits k resident CTAs per SM: one row
    less would exceed k x sms."""
    strips = -(-nx // (threads - 6))
    ctas = lambda h: strips * -(-ny // h)
    hs = autotune.balanced_rows(nx, ny, threads, sms)
    assert hs and len(set(hs)) == len(hs)
    for h in hs:
        k = next(k for k in range(1, autotune.MAX_CTAS_PER_SM + 1) if ctas(h) <= k * sms)
        assert h == 1 or ctas(h - 1) > k * sms


def test_sim_candidates_on_the_splash_grid(autotune):
    """On 2048 x 512 with 152 SMs the candidates include the one-wave heights measured fastest
    (128 x 15: 595 CTAs for 608 slots; 128 x 20: 442 CTAs, three per SM), never a zero height
    (which the library reads as 'keep the current one'), and no duplicates."""
    c = autotune.sim_candidates(2048, 512, 152)
    assert (128, 15) in c and (128, 20) in c and (256, 16) in c
    assert all(r >= 1 for _, r in c) and len(set(c)) == len(c)
