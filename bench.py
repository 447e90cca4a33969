#!/usr/bin/env python
"""Throughput of the two-distribution D2Q9 multiphase LBM step on GB300 (MLUPS, % of HBM roofline).

Workload: droplet splashing on a thin film, 2048 x 512, walls on y, rho 1:0.001, Re 500, We 8000
(the single-simulation configuration whose grid exceeds L2, on which the HBM-roofline figure is
quoted).  A bench step is one time step of the whole path (pull-gather, moments, mu, gradients,
forcing, both collisions, stores) over the grid.  Under the central-difference scheme this
configuration leaves the finite range after ~11 steps, so the state is re-initialised from the
workload's initial fields every 8 steps, outside the timed region: every timed step acts on a
finite state.  L2 is flushed between timed steps (a 512 MB write, then a 512 MB read so that the
flush's own dirty lines are written back before the step, not during it); each step is timed alone with
CUDA events on the simulation's stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (torchrun): independent replicas, one per GPU, no collective on the data path
(``scaling: weak``); value = all ranks' lattice updates / max-over-ranks time.
``--impl reference``: the FP64 CPU oracle on the host cores (rank 0 only), same metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

B_MIN_FP32 = 144          # bytes per lattice update: 2 distributions x 9 x (read + write) x 4 B
REINIT_EVERY = 8
KERNEL_SOURCES = ("paper_1110_5004_gb300/csrc/lbm_device.cuh", "paper_1110_5004_gb300/csrc/lbm_kernels.cu")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tile", default="", help="threads,rows of the step kernel (default: autotuned)")
    ap.add_argument("--e2e-iters", type=int, default=20)
    ap.add_argument("--e2e-jobs", type=int, default=4, help="simulations (streams) in flight in the e2e leg")
    ap.add_argument("--cpu-steps", type=int, default=480,
                    help="oracle steps for the CPU baseline sample on the splash (~10 s); scaled by cells")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--quick", action="store_true", help="main line only (no batch / serving legs)")
    ap.add_argument("--workload", default="splash", choices=["splash", "large"],
                    help="main-line workload: the 2048x512 splash, or the 4096x4096 periodic static drop")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16", "bf16"],
                    help="population storage of the main line (16-bit forms keep FP32 arithmetic)")
    ap.add_argument("--no-flush", action="store_true",
                    help="no L2 flush between timed steps (for DRAM-traffic captures of consecutive steps)")
    ap.add_argument("--batch-sims", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=2000)
    ap.add_argument("--serve-requests", type=int, default=256)
    ap.add_argument("--serve-step-scale", type=float, default=0.2)
    return ap.parse_args()


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def workload(name="splash"):
    import workloads as W
    if name == "large":
        return W.static_droplet(nx=4096, ny=4096, R=600.0)   # 2.4 GB of populations, far beyond L2
    return W.splash()


def kernel_hash():
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def traffic_per_launch(w):
    """DRAM bytes per step-kernel launch from the committed ncu summary of this workload, if it was
    taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    for rec in d if isinstance(d, list) else [d]:          # one record per profiled workload
        if rec.get("kernel_hash") == kernel_hash() and rec.get("workload") == w.name:
            return rec["dram_bytes_per_lu"] * w.cells
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 20 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None
        self.first = 0          # index of the first sample taken inside the timed region

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi takes a moment to start: let it deliver a sample before the timed
            # region begins (bounded wait), and count only the samples taken after that
            deadline = time.perf_counter() + 3.0
            while not self.lines and time.perf_counter() < deadline and self.proc.poll() is None:
                time.sleep(0.01)
            self.first = len(self.lines)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.t is not None:
                self.t.join(timeout=2)

    def summary(self):
        rows = []
        lines = self.lines[self.first:] or self.lines[-1:]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5], parts[6], parts[7], parts[8]))
            except ValueError:
                continue
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), r[2:]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


def replica_throughput(local_seconds, updates_per_rank, world, device=None):
    """Whole-job throughput of N independent replicas: every rank did the same work, the job
    took as long as the slowest rank (max over ranks), value = all ranks' updates / that time."""
    import torch
    import torch.distributed as dist
    slowest = float(local_seconds)
    if world > 1:
        t = torch.tensor([slowest], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        slowest = float(t.item())
    return world * updates_per_rank / slowest / 1e6, slowest


def cpu_baseline(w, steps):
    """The FP64 oracle, as it stands, on the host cores: `steps` steps of the workload with the
    same re-initialisation cadence."""
    import oracle
    s = oracle.Sim.from_workload(w)
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        if done % REINIT_EVERY == 0 and done:
            s.init_fields(w.phi0, w.ux0, w.uy0, w.p0)
        n = min(REINIT_EVERY - done % REINIT_EVERY, steps - done)
        s.step(n)
        done += n
    dt = time.perf_counter() - t0
    cores = oracle.num_threads()
    # the same oracle on one core, over a shorter sample
    one_steps = max(1, steps // 16)
    oracle.set_threads(1)
    try:
        s.init_fields(w.phi0, w.ux0, w.uy0, w.p0)
        t1 = time.perf_counter()
        s.step(one_steps)
        dt1 = time.perf_counter() - t1
    finally:
        oracle.set_threads(cores)
    return {"value": w.cells * steps / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": "%d FP64 oracle steps of %s (%d cells), re-initialised every %d steps, %.1f s"
                      % (steps, w.name, w.cells, REINIT_EVERY, dt),
            "single_core_mlups": w.cells * one_steps / dt1 / 1e6,
            "single_core_sample": "%d steps on one core, %.1f s" % (one_steps, dt1)}


def batch_leg(args, lbm, torch):
    """Ragged batch of independent droplets (256 sims, grids 64^2..512^2, aspect 1..4, seed 1234):
    aggregate MLUPS of the persistent graph-replayed batch vs the same sims stepped back to back
    with the plain stepper; the batch kernel's tile shape is autotuned on the mix."""
    import workloads as W
    from paper_1110_5004_gb300 import autotune
    ws = W.ragged_batch(n=args.batch_sims, steps=args.batch_steps)
    cells = sum(w.cells for w in ws)
    stream = torch.cuda.current_stream()
    out = {"sims": len(ws), "steps": args.batch_steps, "cells": cells,
           "workload": "c4 ragged batch, seed 1234"}
    for st, name in ((0, "fp32"), (1, "fp16"), (2, "bf16")):
        sims = [lbm.Sim.from_workload(w, storage=st, stream=stream) for w in ws]
        b = lbm.Batch(stream=stream)
        for s in sims:
            b.add(s)
        tile = autotune.tune_batch(b, reps=2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.step(args.batch_steps)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ok = [s.diagnostics()["finite"] for s in sims]
        cells_ok = sum(w.cells for w, f in zip(ws, ok) if f)
        out[name] = {"aggregate_mlups": cells * args.batch_steps / dt / 1e6, "seconds": dt,
                     "tile": list(tile[:2]), "finite_at_end": int(sum(ok)),
                     "mlups_finite": cells_ok * args.batch_steps / dt / 1e6}
        b.close()
        for s in sims:
            s.close()
    out["back_to_back_fp32_mlups"] = None
    out["accuracy"] = {"fp32": "FP32 parity with the FP64 oracle (1e-5)",
                       "fp16": "within the reduced-storage bound (phi 1e-3; drift and centroid velocity 0.5 %)",
                       "bf16": "within the reduced-storage bound (stochastic rounding to BF16; falling drop "
                               "0.05 % in centroid velocity, 3.3e-4 in phi)"}
    out["finite_note"] = ("members at density ratios 100 and 1000 leave the finite range under this "
                          "scheme; mlups_finite counts only the members finite after the run")
    return out


def batch_leg_b2b(args, lbm, torch, ws):
    stream = torch.cuda.current_stream()
    total = 0.0
    for w in ws:
        s = lbm.Sim.from_workload(w, stream=stream)
        torch.cuda.synchronize()
        ts = time.perf_counter()
        s.step(args.batch_steps)
        torch.cuda.synchronize()
        total += time.perf_counter() - ts
        s.close()
    return total


def serve_leg(args, lbm, torch):
    """Poisson stream of falling-droplet requests (seed 5678, 50 req/s, grids 128x256..1024x4096,
    density ratio 10..1000), step counts scaled by --serve-step-scale so the run stays bounded:
    continuous batching under a 120 GB budget vs back-to-back plain runs, both in real time."""
    import workloads as W
    from paper_1110_5004_gb300 import serve
    reqs = [serve.Request(r.rid, r.workload, r.workload.steps, r.arrival_s)
            for r in W.serving_stream(n=args.serve_requests, step_scale=args.serve_step_scale)]
    srv = serve.Server(budget_bytes=120 * 10 ** 9, chunk_steps=200, check_steps=400)
    t0 = time.perf_counter()
    res = srv.run(reqs)
    wall = time.perf_counter() - t0
    served = serve.summarize(res, wall)
    served["max_concurrent"] = srv.max_concurrent
    srv.close()
    t0 = time.perf_counter()
    res_p = serve.run_plain(reqs, check_every_steps=400)
    plain = serve.summarize(res_p, time.perf_counter() - t0)
    return {"workload": "c5 Poisson 50 req/s, seed 5678, %d requests, steps x %g"
                        % (len(reqs), args.serve_step_scale),
            "served": served, "plain_back_to_back": plain}


def other_grids(lbm, torch, peak):
    """Secondary lines: a 4096 x 4096 periodic static drop (2.4 GB ping-pong, far above L2) and the
    L2-resident c1 / c2 grids, each on the kernel the library picks by default, timed over
    consecutive steps (no flush: the large grid does not fit in L2, the small ones are labelled
    L2-resident).  The small grids run the tile kernel; for them the row march is timed too, on
    its autotuned tile in the same run, and the ratio is reported."""
    import workloads as W
    from paper_1110_5004_gb300 import autotune
    stream = torch.cuda.current_stream()

    def time_steps(sim, w, steps):
        sim.init_fields(w.phi0, w.ux0, w.uy0, w.p0)
        sim.step(3)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.step(steps)
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) * 1e-3 / steps

    out = {}
    for key, w, steps, label in (("large_grid", W.static_droplet(nx=4096, ny=4096, R=600.0), 20, "exceeds L2"),
                                 ("c1", W.static_droplet(), 400, "L2-resident"),
                                 ("c2", W.falling_droplet(), 40, "L2-resident; re-initialised before timing")):
        sim = lbm.Sim.from_workload(w, stream=stream)
        # the kernel the library picks by default; the row-march tile shape does not apply to the
        # small-grid tile kernel
        small = sim.active_kernel == lbm.LBM_KERNEL_TILES
        t_, r_ = (0, 0) if small else autotune.tune_sim(sim)[:2]
        dt = time_steps(sim, w, steps)
        sim.close()
        mlups = w.cells / dt / 1e6
        out[key] = {"workload": w.name, "cells": w.cells, "mlups": mlups, "us_per_step": dt * 1e6,
                    "hbm_frac_of_measured": B_MIN_FP32 * mlups * 1e6 / (peak * 1e9),
                    "kernel": "tiles (16 x 8 cells per CTA)" if small else "rows",
                    "tile": None if small else [t_, r_], "note": label}
        if key != "large_grid":   # the other kernel on the same grid, same run
            if small:
                rows = lbm.Sim.from_workload(w, stream=stream, kernel=lbm.LBM_KERNEL_ROWS)
                rt, rr = autotune.tune_sim(rows)[:2]
                drow = time_steps(rows, w, steps)
                rows.close()
                out[key].update({"rows_us_per_step": drow * 1e6, "rows_tile": [rt, rr],
                                 "speedup_vs_rows": drow / dt})
            else:
                tiles = lbm.Sim.from_workload(w, stream=stream, kernel=lbm.LBM_KERNEL_TILES)
                dtile = time_steps(tiles, w, steps)
                tiles.close()
                out[key].update({"tiles_us_per_step": dtile * 1e6, "speedup_vs_tiles": dtile / dt})
    return out


def storage16_leg(lbm, torch, w, peak, flush_l2, steps=48):
    """c3 with 16-bit population storage (FP16 and BF16 deviations from the lattice weights, FP32
    arithmetic), timed like the main line: autotuned tile, L2 flushed before every timed step,
    re-initialised every REINIT_EVERY steps outside the timed region.  The roofline is taken
    against 72 B per lattice update (half the FP32 minimum)."""
    from paper_1110_5004_gb300 import autotune
    stream = torch.cuda.current_stream()
    dev0 = [torch.from_numpy(getattr(w, k)).cuda() for k in ("phi0", "ux0", "uy0", "p0")]
    out = {}
    for name, st in (("fp16", 1), ("bf16", 2)):
        sim = lbm.Sim.from_workload(w, stream=stream, storage=st)
        t_, r_, _ = autotune.tune_sim(sim, reps=3)
        for i in range(2 * REINIT_EVERY):
            if i % REINIT_EVERY == 0:
                sim.init_fields(*dev0)
            sim.step(1)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            if i % REINIT_EVERY == 0:
                sim.init_fields(*dev0)
            flush_l2(i)
            ev[i][0].record(stream)
            sim.step(1)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        dt = sum(a.elapsed_time(b) for a, b in ev) * 1e-3 / steps
        mlups = w.cells / dt / 1e6
        out[name] = {"mlups": mlups, "us_per_step": dt * 1e6, "tile": [t_, r_],
                     "bytes_per_lu_algorithmic": B_MIN_FP32 // 2,
                     "hbm_frac_of_measured": (B_MIN_FP32 // 2) * mlups * 1e6 / (peak * 1e9)}
        sim.close()
    out["workload"] = w.name
    out["l2"] = "flushed between timed steps, as the main line"
    out["accuracy"] = {"fp16": "within the reduced-storage bound (phi 1e-3 of the FP64 oracle)",
                       "bf16": "within the reduced-storage bound (stochastic rounding to BF16)"}
    return out


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    w = workload(args.workload)
    import oracle
    res = []
    s = oracle.Sim.from_workload(w)
    total_steps = args.warmup + args.steps
    for i in range(total_steps):
        if i % REINIT_EVERY == 0 and i:
            s.init_fields(w.phi0, w.ux0, w.uy0, w.p0)
        t0 = time.perf_counter()
        s.step(1)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            res.append(dt)
    tot = sum(res)
    value = w.cells * len(res) / tot / 1e6
    line = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot / len(res) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": w.name, "grid": [w.nx, w.ny], "reinit_every": REINIT_EVERY},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "each step one FP64 oracle step of %s" % w.name},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = env_rank()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1110_5004_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    import paper_1110_5004_gb300 as lbm

    w = workload(args.workload)
    stream = torch.cuda.current_stream()
    tile = tuple(int(v) for v in args.tile.split(",")) if args.tile else None
    storage = {"fp32": 0, "fp16": 1, "bf16": 2}[args.storage]
    sim = lbm.Sim.from_workload(w, stream=stream, tile=tile, storage=storage)
    tile_how = "given"
    if tile is None:
        # tile shape measured on this device (cached per device, grid class and kernel source);
        # the tuning steps run before warm-up and the state is re-initialised afterwards
        from paper_1110_5004_gb300 import autotune
        t_, r_, _ = autotune.tune_sim(sim)
        tile, tile_how = (t_, r_), "autotuned"
    dev0 = [torch.from_numpy(getattr(w, k)).cuda() for k in ("phi0", "ux0", "uy0", "p0")]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    clean = torch.ones(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    sink = torch.empty((), dtype=torch.float32, device="cuda")

    def flush_l2(i):
        flush.fill_(float(i))              # evicts the state from L2
        torch.sum(clean, dim=0, out=sink)  # evicts (writes back) the fill's dirty lines

    init_launches = [0]                    # launches of the re-initialisations (not step kernels)

    def reinit():
        l0 = sim.launch_count
        sim.init_fields(*dev0)
        init_launches[0] += sim.launch_count - l0

    for i in range(args.warmup):
        if i % REINIT_EVERY == 0:
            reinit()
        sim.step(1)
    torch.cuda.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = sim.launch_count
    init_launches[0] = 0
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            if i % REINIT_EVERY == 0:
                reinit()
            if not args.no_flush:
                flush_l2(i)
            ev0[i].record(stream)
            sim.step(1)
            ev1[i].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches = sim.launch_count - launches0 - init_launches[0]
    per_step = [a.elapsed_time(b) * 1e-3 for a, b in zip(ev0, ev1)]
    value, total = replica_throughput(sum(per_step), w.cells * args.steps, world, device="cuda")
    mean_step = sum(per_step) / len(per_step)
    peak, peak_kind = measured_peaks()
    # 16-bit storage halves the populations' bytes; f_0 stays a float (76 B moved per update)
    b_min = B_MIN_FP32 if storage == 0 else B_MIN_FP32 // 2
    achieved = b_min * w.cells / mean_step / 1e9
    tr = traffic_per_launch(w) if storage == 0 else None   # the record is of the FP32 step
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": tr, "peak_kind": peak_kind,
                "bytes_per_lu_algorithmic": b_min, "bytes_per_lu_design": 152 if storage == 0 else 76,
                "kernel": "k_tiles<MODE_STEP> (fused gather/moments/mu/forcing/collide/store)"}

    # end to end through the C ABI with pinned host buffers: upload the initial fields, advance
    # REINIT_EVERY steps, read the five moment fields back
    h_in = [torch.from_numpy(getattr(w, k)).pin_memory() for k in ("phi0", "ux0", "uy0", "p0")]
    h_out = {k: torch.empty((w.ny, w.nx), dtype=torch.float32).pin_memory() for k in ("phi", "rho", "ux", "uy", "p")}
    h_in_np = [t.numpy() for t in h_in]
    h_out_np = {k: v.numpy() for k, v in h_out.items()}

    def e2e_iter():
        sim.init_fields(*h_in_np)
        sim.step(REINIT_EVERY)
        sim.moments(h_out_np)

    # the same work as several jobs in flight (--e2e-jobs): one simulation per stream, each driven
    # by its own host thread through the packed calls (one upload and one download per
    # iteration), so that one job's host copies overlap the others' steps
    jobs = max(1, args.e2e_jobs)
    h_block = torch.from_numpy(np.stack([getattr(w, k) for k in ("phi0", "ux0", "uy0", "p0")])).pin_memory().numpy()
    h_res = [torch.empty((5, w.ny, w.nx), dtype=torch.float32).pin_memory().numpy() for _ in range(jobs)]
    sims2 = [sim] + [lbm.Sim.from_workload(w, stream=torch.cuda.Stream(), tile=tile, storage=storage)
                     for _ in range(jobs - 1)]

    def e2e_job(j, iters):
        s = sims2[j]
        for _ in range(iters):
            s.init_fields_packed(h_block)
            s.step(REINIT_EVERY)
            s.moments_packed(h_res[j])

    def e2e_pipelined(iters):
        share = [iters // jobs + (1 if j < iters % jobs else 0) for j in range(jobs)]
        th = [threading.Thread(target=e2e_job, args=(j, n)) for j, n in enumerate(share)]
        for t_ in th:
            t_.start()
        for t_ in th:
            t_.join()

    e2e_value = e2e_serial = None
    if args.e2e_iters > 0:
        for _ in range(2):
            e2e_iter()
        e2e_pipelined(4)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_iters):
            e2e_iter()
        torch.cuda.synchronize()
        e2e_serial, _ = replica_throughput(time.perf_counter() - t0, w.cells * REINIT_EVERY * args.e2e_iters,
                                           world, device="cuda")
        assert np.isfinite(h_out_np["phi"]).all(), "non-finite state inside the re-initialisation window"
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_pipelined(args.e2e_iters)
        torch.cuda.synchronize()
        e2e_value, _ = replica_throughput(time.perf_counter() - t0, w.cells * REINIT_EVERY * args.e2e_iters,
                                          world, device="cuda")
        assert all(np.isfinite(r[0]).all() for r in h_res), "non-finite state inside the re-initialisation window"

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(w, max(REINIT_EVERY, args.cpu_steps * 2048 * 512 // w.cells))

    batch = serving = others = st16 = None
    if not args.quick:
        st16 = storage16_leg(lbm, torch, w, peak, flush_l2)
        others = other_grids(lbm, torch, peak)
        import workloads as W
        batch = batch_leg(args, lbm, torch)
        ws = W.ragged_batch(n=args.batch_sims, steps=args.batch_steps)
        b2b = batch_leg_b2b(args, lbm, torch, ws)
        batch["back_to_back_fp32_mlups"] = batch["cells"] * args.batch_steps / b2b / 1e6
        serving = serve_leg(args, lbm, torch)

    if rank == 0:
        line = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": w.name, "grid": [w.nx, w.ny], "cells": w.cells, "storage": args.storage,
                           "l2": "flushed between timed steps (512 MB write, then 512 MB read); inputs %d MB"
                                 % round(76 * w.cells / 1e6),
                           "reinit_every": REINIT_EVERY, "tile": list(tile), "tile_choice": tile_how,
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": roofline,
                "hbm_roofline_frac_of_measured": achieved / peak,
                "e2e": {"value": e2e_value, "unit": "MLUPS",
                        "h2d_bytes_per_step": 4 * 4 * w.cells // REINIT_EVERY,
                        "d2h_bytes_per_step": 5 * 4 * w.cells // REINIT_EVERY,
                        "what": "per iteration: lbm_init_fields_packed from a pinned host block (4 fields), "
                                "lbm_step(%d), lbm_moments_packed into a pinned host block (5 fields); %d "
                                "simulations on %d streams, each driven by its own host thread; bytes shown "
                                "per LBM step" % (REINIT_EVERY, jobs, jobs),
                        "serial_value": e2e_serial,
                        "serial_what": "one simulation, per-field lbm_init_fields / lbm_moments, iterations "
                                       "back to back"},
                "gpu_launches": launches,
                "clocks": clk.summary(),
                "cpu_baseline": cpu,
                "batch": batch,
                "serving": serving,
                "storage16": st16,
                "other_grids": others}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
