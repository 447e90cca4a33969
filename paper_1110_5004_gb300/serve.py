"""Continuous-batching server for simulation requests.

Requests (a workload and a step count) arrive over time.  Admitted requests keep their f/g
state resident on the device.  Members smaller than `solo_cells` share one ragged batch: each
round advances them by one chunk of steps (replays of one captured 16-step graph, one persistent
launch per step over the tiles of all of them).  Larger members step alone with the
single-simulation kernels, each on a stream of its own, so that their kernels run concurrently
and fill each other's idle SMs.  Each round
  - launches every member's chunk, then, while that runs on the GPU,
  - admits waiting requests in order of priority, then arrival, while the device-memory budget,
    the member cap and the cap on lattice cells in flight allow (a request larger than the whole
    budget is rejected at once; the cell cap never blocks the only request).  A new member is
    created (stream-ordered allocation), initialised or restored on an upload stream, so its
    host copies overlap the running round; it joins at the next round,
  - preempts: when the request at the head of the queue does not fit and members of lower
    priority are running, the fewest of them needed (lowest priority, latest admitted first) are
    evicted -- their state checkpointed to host memory (lbm_checkpoint) and their device memory
    freed -- and queued again; on readmission the state is restored (lbm_restore), so an evicted
    request ends bitwise where an uninterrupted run ends,
  - retires members that reached their step count (FP64 diagnostics and, optionally, the
    moment fields copied back to the host; the member's device memory is freed),
  - retires members whose state stopped being finite (failure detection, LBM_ERR_DIVERGED).
Latency is measured from arrival to the result being on the host.  `run_plain` serves the same
stream back to back, one plain simulation at a time, as the baseline.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Dict, List, Optional

import numpy as np

from . import LBM_FP32, Batch, Sim, device_bytes


@dataclasses.dataclass
class Request:
    rid: int
    workload: object          # workloads.Workload
    steps: int
    arrival_s: float = 0.0
    storage: int = LBM_FP32
    priority: int = 0         # higher is more urgent; may preempt running lower priorities


@dataclasses.dataclass
class Result:
    rid: int
    status: str               # "done" | "diverged" | "rejected" | "cancelled"
    steps_done: int
    arrival_s: float
    admit_s: Optional[float]
    finish_s: float
    diagnostics: Optional[dict] = None
    fields: Optional[Dict[str, np.ndarray]] = None
    evictions: int = 0

    @property
    def latency_s(self):
        return self.finish_s - self.arrival_s


def percentile(xs, q):
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else float("nan")


def summarize(results: List[Result], wall_s: float) -> dict:
    """Counts, p50/p99 latency of the requests that ran (done or diverged), and throughput: over
    every lattice update performed (`mlups`), and over those of the requests that finished with a
    finite state only (`mlups_finite`; a diverged request's updates up to its detection are work
    without a usable result)."""
    done = [r for r in results if r.status == "done"]
    lat = [r.latency_s for r in results if r.status in ("done", "diverged")]
    lu = sum(r.steps_done * r.diagnostics_cells for r in results if hasattr(r, "diagnostics_cells"))
    lu_done = sum(r.steps_done * r.diagnostics_cells for r in done if hasattr(r, "diagnostics_cells"))
    ok = wall_s > 0
    return {"requests": len(results), "done": len(done),
            "diverged": sum(r.status == "diverged" for r in results),
            "rejected": sum(r.status == "rejected" for r in results),
            "p50_s": percentile(lat, 50), "p99_s": percentile(lat, 99), "wall_s": wall_s,
            "lattice_updates": lu, "mlups": lu / wall_s / 1e6 if ok else float("nan"),
            "lattice_updates_finite": lu_done, "mlups_finite": lu_done / wall_s / 1e6 if ok else float("nan")}


class _Pending:
    """A queued request: new, or evicted with its checkpoint."""

    def __init__(self, req: Request, check_steps: int):
        self.req = req
        self.remaining = req.steps
        self.next_check = check_steps
        self.ckpt = None          # host checkpoint of an evicted run
        self.admit_s = None       # first admission
        self.evictions = 0
        self.seq = 0              # admission order, to pick the latest-admitted victim

    def key(self):
        return (-self.req.priority, self.req.arrival_s, self.req.rid)


class _Member:
    def __init__(self, pend: _Pending, sim: Sim, slot: int, solo: bool = False):
        self.pend, self.req, self.sim, self.slot, self.solo = pend, pend.req, sim, slot, solo

    @property
    def remaining(self):
        return self.pend.remaining

    @remaining.setter
    def remaining(self, v):
        self.pend.remaining = v

    @property
    def next_check(self):
        return self.pend.next_check

    @next_check.setter
    def next_check(self, v):
        self.pend.next_check = v

    @property
    def admit_s(self):
        return self.pend.admit_s


class Server:
    def __init__(self, budget_bytes: int, max_members: int = 256, chunk_steps: int = 200,
                 check_steps: int = 200, keep_fields: bool = False, stream=None, tile=None,
                 max_cells: int = 4 << 20, solo_cells: int = 1 << 16, solo_streams: int = 8):
        import torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        # creation, initial state and restores of new members (without a device: the server stream)
        self.upload = torch.cuda.Stream() if torch.cuda.is_available() else self.stream
        self.budget = int(budget_bytes)
        self.batch = Batch(budget_bytes=self.budget, stream=self.stream)
        if tile is not None:
            self.batch.set_tile(*tile)
        self.max_members = max_members
        # lattice cells in flight that already fill the device: admitting beyond them only
        # stretches every member's latency (processor sharing) without adding throughput
        self.max_cells = max_cells
        # a member of at least this many cells steps alone, with the single-simulation kernels
        # (the small-grid tile kernel up to 512K cells, the row march above), on a stream of its
        # own; smaller members share the batch.  On the c5 stream, 64K cells and 8 streams served
        # 23.1 GLUPS against 22.0 with a 1M threshold and 4 streams (256 requests).
        self.solo_cells = solo_cells
        self.solo_bytes = 0
        self._solo_key = 0
        # solo members step on streams of their own, so that one member's last CTAs of a step
        # share the device with the next launches of the others
        self.solo_streams = ([torch.cuda.Stream() for _ in range(solo_streams)] if torch.cuda.is_available()
                             else [self.stream])
        self.chunk = chunk_steps
        self.check_steps = check_steps     # a member is checked for divergence every this many steps
        self.keep_fields = keep_fields
        self.cancelled = set()
        self.max_concurrent = 0
        self.max_bytes = 0                 # peak device bytes held by members
        self.rounds = 0
        self.evictions = 0
        self._seq = 0

    def cancel(self, rid: int):
        self.cancelled.add(rid)

    def _bytes(self):
        return self.batch.bytes + self.solo_bytes

    def _release(self, m: _Member):
        if m.solo:
            self.solo_bytes -= device_bytes(m.req.workload.nx, m.req.workload.ny, m.req.storage)
        else:
            self.batch.remove(m.slot)

    def _finish(self, m: _Member, status: str, now: float, results: List[Result]):
        diag = m.sim.diagnostics()
        fields = m.sim.moments() if self.keep_fields and status == "done" else None
        self._release(m)
        m.sim.close()
        r = Result(m.req.rid, status, m.req.steps - m.remaining, m.req.arrival_s, m.admit_s, now(), diag, fields,
                   m.pend.evictions)
        r.diagnostics_cells = m.req.workload.cells
        results.append(r)

    def _fits(self, r: Request, need: int, active) -> bool:
        cells = sum(m.req.workload.cells for m in active.values())
        return (self._bytes() + need <= self.budget and len(active) < self.max_members and
                (not active or cells + r.workload.cells <= self.max_cells))

    def _victims(self, r: Request, need: int, active):
        """Fewest lower-priority members whose eviction lets r in (lowest priority, latest
        admitted first), or None."""
        cands = sorted((m for m in active.values() if m.req.priority < r.priority),
                       key=lambda m: (m.req.priority, -m.pend.seq))
        chosen, bytes_, count, cells = [], self._bytes(), len(active), \
            sum(m.req.workload.cells for m in active.values())
        for m in cands:
            chosen.append(m)
            bytes_ -= device_bytes(m.req.workload.nx, m.req.workload.ny, m.req.storage)
            count -= 1
            cells -= m.req.workload.cells
            if bytes_ + need <= self.budget and count < self.max_members and \
                    (count == 0 or cells + r.workload.cells <= self.max_cells):
                return chosen
        return None

    def _evict(self, m: _Member):
        self._release(m)
        m.pend.ckpt = m.sim.checkpoint()
        m.sim.close()
        m.pend.evictions += 1
        self.evictions += 1


    def _admit(self, waiting, active, results, now):
        """Admission in priority order, preempting lower priorities when needed.  A new member is
        created and initialised (or restored from its checkpoint) on the upload stream, so that
        this runs while a round is on the GPU, then added to the batch and moved to the server
        stream."""
        while waiting:
            w = waiting[0]
            r = w.req
            need = device_bytes(r.workload.nx, r.workload.ny, r.storage)
            if need > self.budget:
                waiting.pop(0)
                results.append(Result(r.rid, "rejected", 0, r.arrival_s, None, now()))
                continue
            if not self._fits(r, need, active):
                victims = self._victims(r, need, active)
                if victims is None:
                    break
                for m in victims:
                    del active[m.slot]
                    self._evict(m)
                    waiting.append(m.pend)
                waiting.sort(key=_Pending.key)
                continue
            if w.ckpt is not None:
                sim = Sim.from_workload(r.workload, storage=r.storage, stream=self.upload, init=False)
                sim.restore(w.ckpt)
            else:
                sim = Sim.from_workload(r.workload, storage=r.storage, stream=self.upload)
            solo = r.workload.cells >= self.solo_cells
            if solo:
                self._solo_key -= 1
                slot = self._solo_key
                self.solo_bytes += need
                sim.set_stream(self.solo_streams[-slot % len(self.solo_streams)])
            else:
                slot = self.batch.try_add(sim)   # waits for the upload stream only
                if slot is None:            # the library's own budget check agrees with ours
                    sim.close()
                    break
                sim.set_stream(self.stream)
            waiting.pop(0)
            w.ckpt = None
            if w.admit_s is None:
                w.admit_s = now()
            self._seq += 1
            w.seq = self._seq
            active[slot] = _Member(w, sim, slot, solo)

    def run(self, requests: List[Request], realtime: bool = True) -> List[Result]:
        """Serve `requests` (arrival times in seconds from the start).  With realtime=False the
        arrival clock jumps to the next arrival whenever the device would otherwise idle."""
        pending = sorted(requests, key=lambda r: r.arrival_s)
        waiting: List[_Pending] = []
        active: Dict[int, _Member] = {}
        results: List[Result] = []
        t0 = time.perf_counter()
        offset = [0.0]

        def now():
            return time.perf_counter() - t0 + offset[0]

        while pending or waiting or active:
            t = now()
            while pending and pending[0].arrival_s <= t:
                waiting.append(_Pending(pending.pop(0), self.check_steps))
            waiting.sort(key=_Pending.key)
            # cancellations
            for w in [w for w in waiting if w.req.rid in self.cancelled]:
                waiting.remove(w)
                results.append(Result(w.req.rid, "cancelled", w.req.steps - w.remaining, w.req.arrival_s, w.admit_s,
                                      now(), evictions=w.evictions))
            for m in [m for m in active.values() if m.req.rid in self.cancelled]:
                del active[m.slot]
                self._finish(m, "cancelled", now, results)
            if not active:
                self._admit(waiting, active, results, now)
            self.max_concurrent = max(self.max_concurrent, len(active))
            self.max_bytes = max(self.max_bytes, self._bytes())
            if not active:
                if pending:
                    wait = pending[0].arrival_s - now()
                    if wait > 0:
                        if realtime:
                            time.sleep(min(wait, 0.05))
                        else:
                            offset[0] += wait
                continue
            # rounds end where a member finishes or is due for its divergence check
            k = min(self.chunk, min(min(m.remaining, m.next_check - (m.req.steps - m.remaining))
                                    for m in active.values()))
            if any(not m.solo for m in active.values()):
                self.batch.step(k)
            for m in active.values():
                if m.solo:
                    m.sim.step(k)
            self.rounds += 1
            for m in active.values():
                m.remaining -= k
            # admission while the round runs: new members are created, initialised (or restored)
            # and added on the upload stream, and join the batch at the next round
            self._admit(waiting, active, results, now)
            self.max_concurrent = max(self.max_concurrent, len(active))
            self.max_bytes = max(self.max_bytes, self._bytes())
            finished = [m for m in active.values() if m.remaining == 0]
            for m in finished:
                del active[m.slot]
                self._finish(m, "done", now, results)
            for m in list(active.values()):
                done = m.req.steps - m.remaining
                if done >= m.next_check:
                    m.next_check += self.check_steps
                    if not m.sim.diagnostics()["finite"]:
                        del active[m.slot]
                        self._finish(m, "diverged", now, results)
        return sorted(results, key=lambda r: r.rid)

    def close(self):
        self.batch.close()


def run_plain(requests: List[Request], keep_fields: bool = False, stream=None, realtime: bool = True,
              check_every_steps: int = 200) -> List[Result]:
    """Back-to-back baseline: one plain simulation at a time, in arrival order."""
    import torch
    stream = stream if stream is not None else torch.cuda.current_stream()
    results = []
    t0 = time.perf_counter()
    offset = 0.0
    for r in sorted(requests, key=lambda r: r.arrival_s):
        t = time.perf_counter() - t0 + offset
        if r.arrival_s > t:
            if realtime:
                time.sleep(r.arrival_s - t)
            else:
                offset += r.arrival_s - t
        start = time.perf_counter() - t0 + offset
        sim = Sim.from_workload(r.workload, storage=r.storage, stream=stream)
        done, status = 0, "done"
        while done < r.steps:
            n = min(check_every_steps, r.steps - done)
            sim.step(n)
            done += n
            if done < r.steps and not sim.diagnostics()["finite"]:
                status = "diverged"
                break
        diag = sim.diagnostics()
        fields = sim.moments() if keep_fields and status == "done" else None
        sim.close()
        res = Result(r.rid, status, done, r.arrival_s, start, time.perf_counter() - t0 + offset, diag, fields)
        res.diagnostics_cells = r.workload.cells
        results.append(res)
    return sorted(results, key=lambda r: r.rid)
