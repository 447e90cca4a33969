"""Continuous-batching server: admission under a device-memory budget, failure detection,
cancellation, and (on the GPU) every served result equal to the same request run alone."""
import numpy as np
import pytest

import workloads as W


# ----------------------------------------------------------------- host logic with fakes (CPU)

class FakeSim:
    live = 0

    def __init__(self, w, diverge_at=None):
        self.w, self.steps, self.diverge_at = w, 0, diverge_at
        FakeSim.live += 1

    @classmethod
    def from_workload(cls, w, storage=0, stream=None, init=True):
        return cls(w, w.meta.get("diverge_at"))

    def checkpoint(self):
        return {"steps": self.steps}

    def restore(self, ck):
        self.steps = ck["steps"]

    def diagnostics(self):
        ok = self.diverge_at is None or self.steps < self.diverge_at
        return {"finite": int(ok), "step": self.steps}

    def moments(self):
        return {"phi": np.full((self.w.ny, self.w.nx), float(self.steps), np.float32)}

    def set_stream(self, stream):
        pass

    def step(self, k):
        self.steps += k

    def close(self):
        FakeSim.live -= 1


class FakeBatch:
    def __init__(self, budget_bytes=0, stream=None):
        self.budget, self.members, self.bytes, self.history = budget_bytes, {}, 0, []

    def set_tile(self, *a):
        pass

    def try_add(self, sim):
        need = sim.w.nx * sim.w.ny
        if self.bytes + need > self.budget:
            return None
        slot = len(self.members) + len(self.history) * 1000
        while slot in self.members:
            slot += 1
        self.members[slot] = sim
        self.bytes += need
        return slot

    def remove(self, slot):
        sim = self.members.pop(slot)
        self.bytes -= sim.w.nx * sim.w.ny

    def step(self, k):
        self.history.append((k, len(self.members)))
        for s in self.members.values():
            s.steps += k
        FakeClock.t += 1e-4 * k

    def close(self):
        pass


class FakeClock:
    """Time advances only with the batch's steps (0.1 ms per step)."""
    t = 0.0

    @classmethod
    def perf_counter(cls):
        return cls.t

    @staticmethod
    def sleep(dt):
        FakeClock.t += dt


@pytest.fixture
def fake_server(monkeypatch):
    from paper_1110_5004_gb300 import serve
    monkeypatch.setattr(serve, "Sim", FakeSim)
    monkeypatch.setattr(serve, "Batch", FakeBatch)
    monkeypatch.setattr(serve, "device_bytes", lambda nx, ny, st=0: nx * ny)
    monkeypatch.setattr(serve, "time", FakeClock)
    FakeSim.live = 0
    FakeClock.t = 0.0
    return serve


def _req(serve, rid, nx, ny, steps, arrival, **meta):
    w = W.make("r%d" % rid, nx, ny, W.Physical(sigma=0.01, W=4.0), steps, np.zeros((ny, nx)), **meta)
    return serve.Request(rid, w, steps, arrival)


def test_admission_respects_budget_and_order(fake_server):
    serve = fake_server
    reqs = [_req(serve, i, 10, 10, 100 + 50 * i, 0.0) for i in range(5)]
    srv = serve.Server(budget_bytes=250, chunk_steps=60, check_steps=50, stream=0)     # room for two at a time
    res = srv.run(reqs, realtime=False)
    assert [r.status for r in res] == ["done"] * 5
    assert all(r.steps_done == q.steps for r, q in zip(res, reqs))
    assert srv.max_concurrent == 2
    assert max(n for _, n in srv.batch.history) == 2
    assert srv.max_bytes == 200
    # first come first served: admission times are non-decreasing in arrival order
    admits = [r.admit_s for r in res]
    assert admits == sorted(admits)
    assert FakeSim.live == 0                       # every member's memory was released


def test_large_members_step_alone_within_the_budget(fake_server):
    """Members of at least solo_cells cells step alone (their own kernel, not the batch), count
    against the same budget, and finish, diverge and release memory like batch members."""
    serve = fake_server
    reqs = [_req(serve, 0, 20, 20, 200, 0.0),                  # 400 cells: alone
            _req(serve, 1, 10, 10, 150, 0.0),                  # 100 cells: batched
            _req(serve, 2, 20, 20, 300, 0.0, diverge_at=120),  # alone, goes non-finite
            _req(serve, 3, 10, 10, 250, 0.0)]
    srv = serve.Server(budget_bytes=1000, chunk_steps=60, check_steps=60, stream=0, solo_cells=400)
    res = {r.rid: r for r in srv.run(reqs, realtime=False)}
    assert res[0].status == "done" and res[0].steps_done == 200
    assert res[1].status == "done" and res[1].steps_done == 150
    assert res[2].status == "diverged" and res[2].steps_done == 120
    assert res[3].status == "done" and res[3].steps_done == 250
    assert max(n for _, n in srv.batch.history) <= 2          # only the small members batched
    assert srv.max_bytes <= 1000 and srv.solo_bytes == 0 and srv.batch.bytes == 0
    assert FakeSim.live == 0


def test_rejection_divergence_and_cancellation(fake_server):
    serve = fake_server
    reqs = [_req(serve, 0, 10, 10, 300, 0.0),
            _req(serve, 1, 40, 40, 300, 0.0),                 # larger than the whole budget
            _req(serve, 2, 10, 10, 300, 0.0, diverge_at=100),  # goes non-finite
            _req(serve, 3, 10, 10, 300, 0.0)]
    srv = serve.Server(budget_bytes=1000, chunk_steps=50, check_steps=50, stream=0)
    srv.cancel(3)
    res = {r.rid: r for r in srv.run(reqs, realtime=False)}
    assert res[0].status == "done" and res[0].steps_done == 300
    assert res[1].status == "rejected"
    assert res[2].status == "diverged" and res[2].steps_done == 100
    assert res[3].status == "cancelled"
    assert FakeSim.live == 0


def test_priority_preemption_checkpoints_and_resumes(fake_server):
    serve = fake_server
    low = [_req(serve, i, 10, 10, 1000, 0.0) for i in range(3)]
    high = serve.Request(9, _req(serve, 9, 10, 10, 300, 0.0).workload, 300, arrival_s=0.03, priority=5)
    srv = serve.Server(budget_bytes=200, chunk_steps=50, check_steps=100, stream=0)   # two at a time
    res = {r.rid: r for r in srv.run(low + [high], realtime=False)}
    assert all(r.status == "done" for r in res.values())
    assert all(res[i].steps_done == 1000 for i in range(3)) and res[9].steps_done == 300
    assert srv.evictions >= 1 and sum(r.evictions for r in res.values()) == srv.evictions
    assert res[9].evictions == 0
    # the urgent request was admitted soon after it arrived, before the low-priority backlog
    assert res[9].admit_s < 0.04 and res[9].finish_s < res[2].finish_s
    assert srv.max_bytes <= 200
    assert FakeSim.live == 0


def test_no_preemption_among_equal_priorities(fake_server):
    serve = fake_server
    reqs = [_req(serve, i, 10, 10, 400, 0.01 * i) for i in range(4)]
    srv = serve.Server(budget_bytes=200, chunk_steps=50, check_steps=100, stream=0)
    res = srv.run(reqs, realtime=False)
    assert [r.status for r in res] == ["done"] * 4 and srv.evictions == 0


def test_summary_percentiles(fake_server):
    serve = fake_server
    rs = [serve.Result(i, "done", 10, 0.0, 0.0, float(i + 1)) for i in range(100)]
    for r in rs:
        r.diagnostics_cells = 100
    s = serve.summarize(rs, wall_s=10.0)
    assert s["p50_s"] == pytest.approx(50.5) and s["p99_s"] == pytest.approx(99.01)
    assert s["lattice_updates"] == 100 * 10 * 100


# ----------------------------------------------------------------- GPU


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_5004_gb300 import build
    build.build()
    import paper_1110_5004_gb300 as m
    return m


def gpu_stream():
    rng = np.random.default_rng(77)
    reqs = []
    from paper_1110_5004_gb300 import serve
    for i in range(8):
        nx = int(rng.integers(20, 150))
        ny = int(rng.integers(16, 90))
        wall = bool(i % 2)
        w = W.random_small(nx, ny, seed=100 + i, bc_y=W.WALL if wall else W.PERIODIC,
                           gravity=1e-5 if wall else 0.0, remove_Fa=i % 3 == 0)
        reqs.append(serve.Request(i, w, int(rng.integers(40, 260)), arrival_s=0.004 * i,
                                  storage=1 if i == 5 else 0))
    return reqs


@pytest.mark.gpu
@pytest.mark.parametrize("solo_cells", [1 << 20, 4000, 0])
def test_served_results_equal_alone(lbm, solo_cells):
    """Bitwise the results of the same requests run one by one: all batched (1M), the larger ones
    alone on streams of their own next to the batch of the smaller ones (4000), all alone (0)."""
    import dataclasses
    from paper_1110_5004_gb300 import serve
    # all arrive at once, so that their work overlaps however fast each runs
    reqs = [dataclasses.replace(r, arrival_s=0.0) for r in gpu_stream()]
    srv = serve.Server(budget_bytes=1 << 34, chunk_steps=64, keep_fields=True, solo_cells=solo_cells)
    served = srv.run(reqs)
    alone = serve.run_plain(reqs, keep_fields=True)
    assert srv.max_concurrent >= 2                      # work of several requests overlapped
    for a, b in zip(served, alone):
        assert a.status == b.status == "done"
        for k in a.fields:
            assert np.array_equal(a.fields[k], b.fields[k]), (a.rid, k)
    s = serve.summarize(served, wall_s=max(r.finish_s for r in served))
    assert np.isfinite(s["p50_s"]) and np.isfinite(s["p99_s"]) and s["mlups"] > 0
    srv.close()


@pytest.mark.gpu
def test_served_budget_failure_and_cancel(lbm):
    from paper_1110_5004_gb300 import serve
    reqs = gpu_stream()[:5]
    bad = reqs[2].workload
    bad.phi0 = bad.phi0.copy()
    bad.phi0[3, 4] = np.nan                             # fault injected on the host
    need = [lbm.device_bytes(r.workload.nx, r.workload.ny, r.storage) for r in reqs]
    budget = sorted(need)[-1] + sorted(need)[-2]
    huge = serve.Request(99, W.random_small(2000, 2000, seed=1), 10, 0.0)
    srv = serve.Server(budget_bytes=budget, chunk_steps=32, check_steps=32, keep_fields=True)
    srv.cancel(4)
    res = {r.rid: r for r in srv.run(reqs + [huge])}
    assert res[99].status == "rejected"
    assert res[2].status == "diverged"
    assert res[4].status == "cancelled"
    assert 0 < srv.max_bytes <= budget                  # the budget held at every admission
    alone = {r.rid: r for r in serve.run_plain([reqs[0], reqs[1], reqs[3]], keep_fields=True)}
    for rid in (0, 1, 3):
        assert res[rid].status == "done"
        assert np.array_equal(res[rid].fields["phi"], alone[rid].fields["phi"])
    srv.close()


@pytest.mark.gpu
def test_preempted_requests_end_bitwise_as_uninterrupted(lbm, monkeypatch):
    """Low-priority requests evicted to host memory by an urgent one and restored later end
    bitwise where the same requests end run alone without interruption.  The server's clock
    advances with the batch's steps, so the urgent request arrives after 100 steps."""
    from paper_1110_5004_gb300 import serve
    monkeypatch.setattr(serve, "time", FakeClock)
    FakeClock.t = 0.0
    base = gpu_stream()[:4]
    low = [serve.Request(r.rid, r.workload, 400, arrival_s=0.0, storage=r.storage) for r in base[:3]]
    urgent = serve.Request(50, base[3].workload, 200, arrival_s=0.01, priority=3)
    need = {r.rid: lbm.device_bytes(r.workload.nx, r.workload.ny, r.storage) for r in low + [urgent]}
    # room for the largest low request next to the urgent one, not for two low ones next to it
    budget = max(need[r.rid] for r in low) + need[50] + 1000
    srv = serve.Server(budget_bytes=budget, chunk_steps=40, check_steps=80, keep_fields=True)
    step = srv.batch.step

    def timed_step(k):
        step(k)
        FakeClock.t += 1e-4 * k

    srv.batch.step = timed_step
    res = {r.rid: r for r in srv.run(low + [urgent], realtime=False)}
    alone = {r.rid: r for r in serve.run_plain(low + [urgent], keep_fields=True, realtime=False)}
    assert srv.evictions >= 1 and res[50].evictions == 0
    for rid, r in res.items():
        assert r.status == alone[rid].status == "done"
        for k in r.fields:
            assert np.array_equal(r.fields[k], alone[rid].fields[k]), (rid, k)
    srv.close()


@pytest.mark.gpu
@pytest.mark.parametrize("storage,s_form", [(0, 0), (1, 0), (0, 1)])
def test_checkpoint_restore_bitwise(lbm, storage, s_form):
    import dataclasses
    import torch
    w = W.random_small(83, 47, seed=21, bc_y=W.WALL, gravity=1e-5, remove_Fa=1)
    w = dataclasses.replace(w, phys=dataclasses.replace(w.phys, s_form=s_form))
    a = lbm.Sim.from_workload(w, storage=storage)
    a.step(37)
    ck = a.checkpoint()
    assert ck.nbytes == a.checkpoint_bytes
    a.step(41)
    b = lbm.Sim.from_workload(w, storage=storage, init=False)
    b.restore(ck)
    assert b.step_count == 37
    b.step(41)
    ma, mb = a.moments(), b.moments()
    for k in ma:
        assert np.array_equal(ma[k], mb[k]), k
    # device-resident checkpoint buffer
    dev = torch.empty(a.checkpoint_bytes, dtype=torch.uint8, device="cuda")
    a.checkpoint(dev)
    c = lbm.Sim.from_workload(w, storage=storage, init=False)
    c.restore(dev)
    assert c.step_count == 78 and np.array_equal(c.moments()["phi"], ma["phi"])
    # mismatches are rejected and leave the state unchanged
    assert a.device_bytes == lbm.device_bytes(w.nx, w.ny, storage) + (16 * 47 * 96 if s_form else 0)
    other = lbm.Sim.from_workload(W.random_small(84, 47, seed=21), storage=storage)
    before = other.moments()["phi"]
    with pytest.raises(lbm.LBMError):
        other.restore(ck)
    bad = ck.copy()
    bad[0] ^= 0xFF
    with pytest.raises(lbm.LBMError):
        b.restore(bad)
    with pytest.raises(lbm.LBMError):
        b.restore(ck[:100])
    assert np.array_equal(other.moments()["phi"], before)
