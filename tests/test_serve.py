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
    def from_workload(cls, w, storage=0, stream=None):
        return cls(w, w.meta.get("diverge_at"))

    def diagnostics(self):
        ok = self.diverge_at is None or self.steps < self.diverge_at
        return {"finite": int(ok), "step": self.steps}

    def moments(self):
        return {"phi": np.full((self.w.ny, self.w.nx), float(self.steps), np.float32)}

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

    def close(self):
        pass


@pytest.fixture
def fake_server(monkeypatch):
    from paper_1110_5004_gb300 import serve
    monkeypatch.setattr(serve, "Sim", FakeSim)
    monkeypatch.setattr(serve, "Batch", FakeBatch)
    monkeypatch.setattr(serve, "device_bytes", lambda nx, ny, st=0: nx * ny)
    FakeSim.live = 0
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
def test_served_results_equal_alone(lbm):
    from paper_1110_5004_gb300 import serve
    reqs = gpu_stream()
    srv = serve.Server(budget_bytes=1 << 34, chunk_steps=64, keep_fields=True)
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
