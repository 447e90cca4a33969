"""Tile-shape autotuner for the fused step kernel and the batch kernel.

The step kernel's shape is (threads per CTA, rows per CTA).  Threads fix the strip width
(threads - 6 interior columns); rows trade pipeline fill (a segment of h rows runs h + 8 row
iterations, the first and last few with stages idle) for parallelism (one CTA per strip x
segment).  The kernel is bound by instruction issue, so a step lasts as long as the SM with the
most CTAs: besides a fixed list of heights, the candidates include, for k = 1..8 resident CTAs
per SM, the shortest height whose CTA count still fits k x SMs (one row less can add a nearly
empty wave).  The best pair depends on the grid, the storage and the device, so it is
measured: each candidate runs about a millisecond of steps timed with CUDA events on the
simulation's stream, and the fastest is cached per (device, grid class, storage, kernel source)
in a JSON file next to the library (git-ignored).
"""
from __future__ import annotations

import hashlib
import json
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "_autotune_cache.json")
THREADS = (64, 128, 256)
ROWS = (1, 2, 4, 8, 12, 16, 24, 32, 48, 64, 128)
MAX_CTAS_PER_SM = 8
_lock = threading.Lock()


def _kernel_hash():
    h = hashlib.sha256()
    for f in ("lbm_device.cuh", "lbm_kernels.cu", "lbm_batch.cu"):
        with open(os.path.join(HERE, "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def _device_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device()).replace(" ", "_")


def grid_class(nx, ny):
    """Grids of similar shape share a tuned tile: round sizes up to powers of two."""
    def up(v):
        p = 32
        while p < v:
            p *= 2
        return p
    return "%dx%d" % (up(nx), up(ny))


def _load():
    if os.path.exists(CACHE):
        try:
            with open(CACHE) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}
    return {}


def _store(cache):
    tmp = CACHE + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


TUNER_VERSION = "whole-waves-1"   # entries measured over another candidate set are not reused


def _key(kind, nx, ny, storage):
    return "|".join((kind, _device_name(), _kernel_hash(), grid_class(nx, ny), "st%d" % storage, TUNER_VERSION))


def _time(fn, reps, stream):
    import torch
    fn()                                            # warm-up (graph capture, attributes)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / reps


def _sm_count():
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def balanced_rows(nx, ny, threads, sms, max_per_sm=MAX_CTAS_PER_SM):
    """For each k = 1..max_per_sm, the shortest height h whose CTA count strips x ceil(ny / h)
    is at most k x sms (the strip count follows the library's rule: strips of at most
    threads - 6 columns)."""
    strips = -(-nx // (threads - 6))
    out = []
    for k in range(1, max_per_sm + 1):
        segs = (k * sms) // strips
        if segs < 1:
            continue
        h = -(-ny // segs)
        if h not in out:
            out.append(h)
    return out


def sim_candidates(nx, ny, sms):
    """(threads, rows) pairs measured for an nx x ny simulation on a device with `sms` SMs."""
    out = []
    for t in THREADS:
        for r in list(ROWS) + balanced_rows(nx, ny, t, sms):
            if (t, r) not in out:
                out.append((t, r))
    return out


def _reps_for(fn, stream, target_ms=1.0, lo=6, hi=400):
    """Repetitions that make a timed run last about target_ms."""
    one = _time(fn, 2, stream)
    return max(lo, min(hi, int(target_ms / max(one, 1e-4))))


def tune_sim(sim, reps=None, candidates=None, use_cache=True):
    """Measure tile candidates on `sim` (its state advances; re-initialise it afterwards) and
    set the fastest.  Returns (threads, rows, ms per step).  The cache key includes the
    simulation's population storage.  `reps` None: about a millisecond of steps per candidate."""
    import torch
    key = _key("sim", sim.nx, sim.ny, int(sim.params.storage))
    with _lock:
        cache = _load() if use_cache else {}
    if key in cache:
        t, r, ms = cache[key]
        sim.set_tile(t, r)
        return t, r, ms
    stream = torch.cuda.current_stream()
    sim.set_stream(stream)
    best = None
    for t, r in candidates or sim_candidates(sim.nx, sim.ny, _sm_count()):
        sim.set_tile(t, r)
        n = reps if reps else _reps_for(lambda: sim.step(1), stream)
        ms = _time(lambda: sim.step(1), n, stream)
        if best is None or ms < best[2]:
            best = (t, r, ms)
    sim.set_tile(best[0], best[1])
    if use_cache:
        with _lock:
            cache = _load()
            cache[key] = list(best)
            _store(cache)
    return best


BATCH_THREADS = (64, 128, 256)
BATCH_ROWS = (16, 32, 64, 128)


def tune_batch(batch, reps=3, candidates=None):
    """Measure (threads, rows) of the batch kernel on the current membership (members advance).
    Returns (threads, rows, ms per step)."""
    import torch
    stream = torch.cuda.current_stream()
    best = None
    for t, r in candidates or [(t, r) for t in BATCH_THREADS for r in BATCH_ROWS]:
        batch.set_tile(t, r)
        ms = _time(lambda: batch.step(2), reps, stream) / 2      # per step, like best[2]
        if best is None or ms < best[2]:
            best = (t, r, ms)
    batch.set_tile(best[0], best[1])
    return best
