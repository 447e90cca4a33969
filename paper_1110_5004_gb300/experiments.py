"""The paper's two numerical tests at their own sizes, the original scheme against the corrected
one (additional interfacial force removed), advanced side by side on the GPU.

Falling droplet (150 x 450, Eo = 17): the paper reports that the two schemes agree up to
t = 1e4 and then part, the original drop less stretched and lower, with the spread radii 4.1
lattice units apart at t = 1.9e4 (about a quarter of the initial radius).  Splash on a film
(300 x 150, We = 960, Re = 48 and 480): the schemes agree at Re = 48 and differ at Re = 480.

Each run records the FP64 diagnostics (spread radius, liquid centroid and velocity, total phi)
and the largest |F_a,y| of the additional interfacial force F_a = -u s (Eq. 12, evaluated in
both schemes) every `every` steps and, optionally, density and F_a,y fields (the paper's Fig. 3)
at chosen steps; a run that leaves the finite range stops there and reports the step (the
scheme, not the kernel: the FP64 oracle diverges at the same step).

Both tests run under each order-parameter LBE: the equilibrium form with the mu term, and the
forced form (f_form = 1), under which the splash stays finite to the paper's t* = 2.

  python -m paper_1110_5004_gb300.experiments [--out results.json] [--falling-steps 19000]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import Sim

KEYS = ("spread_radius", "centroid_x", "centroid_y", "vel_y", "liquid_area", "sum_phi", "finite")
CONTOUR_LEVEL = 0.55          # the paper's density contours (rho = 0.55, between rho_G = 0.1 and rho_L = 1)


def contour_segments(field, level=CONTOUR_LEVEL):
    """Iso-line field == level by marching squares on the cell-centre grid: an (n, 2, 2) array
    of segments [[x0, y0], [x1, y1]] in lattice units (x along columns, y along rows), each
    endpoint linearly interpolated on a square's edge.  Saddle squares join the corners by the
    sign of the square's mean."""
    f = np.asarray(field, dtype=np.float64) - level
    a, b, c, d = f[:-1, :-1], f[:-1, 1:], f[1:, 1:], f[1:, :-1]   # corners (x,y), (x+1,y), (x+1,y+1), (x,y+1)
    yy, xx = np.mgrid[0:f.shape[0] - 1, 0:f.shape[1] - 1].astype(np.float64)

    def cut(v0, v1):
        den = v0 - v1
        return np.where(den != 0, v0 / np.where(den != 0, den, 1.0), 0.5)

    # edge points: bottom (a-b), right (b-c), top (d-c), left (a-d)
    pts = {"B": np.stack([xx + cut(a, b), yy], -1), "R": np.stack([xx + 1, yy + cut(b, c)], -1),
           "T": np.stack([xx + cut(d, c), yy + 1], -1), "L": np.stack([xx, yy + cut(a, d)], -1)}
    code = (a > 0).astype(int) | ((b > 0).astype(int) << 1) | ((c > 0).astype(int) << 2) | ((d > 0).astype(int) << 3)
    mean_pos = (a + b + c + d) > 0
    table = {1: [("L", "B")], 2: [("B", "R")], 3: [("L", "R")], 4: [("R", "T")], 6: [("B", "T")],
             7: [("L", "T")], 8: [("T", "L")], 9: [("T", "B")], 11: [("T", "R")], 12: [("R", "L")],
             13: [("R", "B")], 14: [("B", "L")]}
    segs = []
    for k, edges in table.items():
        m = code == k
        for e0, e1 in edges:
            segs.append(np.stack([pts[e0][m], pts[e1][m]], 1))
    for k, joined, split in ((5, [("L", "T"), ("B", "R")], [("L", "B"), ("R", "T")]),
                             (10, [("B", "L"), ("T", "R")], [("B", "R"), ("T", "L")])):
        for sel, edges in ((mean_pos, joined), (~mean_pos, split)):
            m = (code == k) & sel
            for e0, e1 in edges:
                segs.append(np.stack([pts[e0][m], pts[e1][m]], 1))
    return np.concatenate(segs, 0) if segs else np.zeros((0, 2, 2))


def liquid_regions(rho, level=CONTOUR_LEVEL, periodic_x=True):
    """Number of connected regions with rho >= level (8-neighbour connectivity, joined across a
    periodic x boundary): the drop, the film and any secondary droplets."""
    from scipy import ndimage
    mask = np.asarray(rho) >= level
    lab, n = ndimage.label(mask, structure=np.ones((3, 3), int))
    if periodic_x and n > 1:
        parent = list(range(n + 1))

        def find(i):
            while parent[i] != i:
                parent[i] = parent[parent[i]]
                i = parent[i]
            return i
        left, right = lab[:, 0], lab[:, -1]
        for y in range(lab.shape[0]):
            for dy in (-1, 0, 1):
                yy = y + dy
                if 0 <= yy < lab.shape[0] and left[y] and right[yy]:
                    parent[find(left[y])] = find(right[yy])
        n = len({find(i) for i in range(1, n + 1)})
    return int(n)


def run_pair(make, steps, every, snapshot_steps=(), stream=None, variants=None):
    """Advance make(remove_Fa=0) and make(remove_Fa=1) for `steps` steps; diagnostics and the
    largest |F_a,y| every `every` steps, density and F_a,y fields at `snapshot_steps`.
    `variants` maps further names to functions of the corrected workload (e.g. another
    definition of the mass defect)."""
    import torch
    stream = stream if stream is not None else torch.cuda.current_stream()
    out = {}
    t0 = time.perf_counter()
    runs = [("original", 0, None), ("corrected", 1, None)] + [(k, 1, f) for k, f in (variants or {}).items()]
    for name, rf, fn in runs:
        w = make(remove_Fa=rf)
        if fn is not None:
            w = fn(w)
        sim = Sim.from_workload(w, stream=stream)
        series = {k: [] for k in ("step",) + KEYS + ("max_abs_fa_y",)}
        snaps = {}
        done = 0
        while True:
            d = sim.diagnostics()
            series["step"].append(done)
            for k in KEYS:
                series[k].append(float(d[k]))
            fa_y = sim.interfacial_force()["fay"]
            series["max_abs_fa_y"].append(float(np.abs(fa_y).max()) if d["finite"] else float("nan"))
            if done in snapshot_steps:
                rho = sim.moments()["rho"]
                snaps[done] = {"rho": rho, "fa_y": fa_y, "contour": contour_segments(rho),
                               "liquid_regions": liquid_regions(rho) if d["finite"] else None}
            if done >= steps or not d["finite"]:
                break
            n = min(every, steps - done)
            sim.step(n)
            done += n
        sim.close()
        out[name] = {"workload": w.name, "series": series, "snapshots": snaps,
                     "diverged_at": None if series["finite"][-1] else series["step"][-1]}
    out["seconds"] = time.perf_counter() - t0
    return out


def difference(res, key="spread_radius", other="corrected"):
    """other - original of one diagnostic at the common steps where both are finite."""
    a, b = res["original"]["series"], res[other]["series"]
    n = min(len(a["step"]), len(b["step"]))
    while n > 1 and not (a["finite"][n - 1] and b["finite"][n - 1]):
        n -= 1
    return np.asarray(a["step"][:n]), np.asarray(b[key][:n]) - np.asarray(a[key][:n])


def _direct_defect(w):
    import dataclasses
    return dataclasses.replace(w, phys=dataclasses.replace(w.phys, s_form=1))


def _with_f_form(w, f_form):
    import dataclasses
    return dataclasses.replace(w, phys=dataclasses.replace(w.phys, f_form=int(f_form)))


def falling_drop(steps=19000, every=100, snapshot_steps=(), stream=None, direct_defect=False, f_form=0):
    """direct_defect: also run the corrected scheme with the mass defect taken directly from the
    stored density and flux (s_form = 1) instead of Eq. 5, to see how F_a depends on it.
    f_form: the order-parameter LBE (0: equilibrium with the mu term, 1: forced form)."""
    import workloads as W
    res = run_pair(lambda remove_Fa: _with_f_form(W.paper_falling_droplet(steps=steps, remove_Fa=remove_Fa), f_form),
                   steps, every, snapshot_steps, stream,
                   {"corrected_direct_s": _direct_defect} if direct_defect else None)
    t, dr = difference(res)
    _, dy = difference(res, "centroid_y")
    r0 = res["original"]["series"]["spread_radius"][0]
    onset = next((int(s) for s, v in zip(t, dr) if abs(v) >= 0.05 * r0), None)
    res["summary"] = {"diverged_at": {k: res[k]["diverged_at"] for k in ("original", "corrected")},
                      "initial_spread_radius": r0,
                      "spread_radius_difference_at_end": float(dr[-1]),
                      "relative_to_initial_radius": float(dr[-1] / r0),
                      "centroid_y_difference_at_end": float(dy[-1]),
                      "onset_step_5pct_of_radius": onset,
                      **({"direct_s_spread_radius_difference_at_end": float(difference(res, other="corrected_direct_s")[1][-1]),
                          "direct_s_centroid_y_difference_at_end":
                              float(difference(res, "centroid_y", other="corrected_direct_s")[1][-1]),
                          "direct_s_diverged_at": res["corrected_direct_s"]["diverged_at"]}
                         if "corrected_direct_s" in res else {}),
                      "paper": "4.1 l.u. at t = 1.9e4 (26 % of the initial radius); parting from t = 1e4"}
    return res


SPLASH_T_STAR = (1.2, 1.8, 2.0)   # the paper's Fig. 2 / Fig. 3 times


def splash(Re, steps=3000, every=50, snapshot_steps=None, stream=None, f_form=0):
    """f_form: the order-parameter LBE (0: equilibrium with the mu term, 1: forced form).
    Snapshots (density, its rho = 0.55 contour, the count of liquid regions, F_a,y) default to
    the paper's t* = 1.2, 1.8 and 2.0 (t* = t U / D, U = 0.04, D = 60)."""
    import workloads as W
    if snapshot_steps is None:
        snapshot_steps = tuple(int(round(ts * 60.0 / 0.04)) for ts in SPLASH_T_STAR)
    snapshot_steps = tuple(s for s in snapshot_steps if s % every == 0 and s <= steps)
    res = run_pair(lambda remove_Fa: _with_f_form(W.paper_splash(Re=Re, steps=steps, remove_Fa=remove_Fa), f_form),
                   steps, every, snapshot_steps, stream)
    t, dr = difference(res)
    # Fig. 3 shows F_a,y of the original scheme at t* = 1.8; report it there, or at the last
    # finite diagnostic before it
    o = res["original"]["series"]
    fig3 = int(round(1.8 * 60.0 / 0.04))
    idx = [i for i, (st, ok) in enumerate(zip(o["step"], o["finite"])) if ok and st <= fig3]
    res["summary"] = {"diverged_at": {k: res[k]["diverged_at"] for k in ("original", "corrected")},
                      "Re": Re, "t_star_per_step": 0.04 / 60.0,
                      "fig3_step": fig3,
                      "max_abs_fa_y_original": {"step": o["step"][idx[-1]], "value": o["max_abs_fa_y"][idx[-1]]}
                      if idx else None,
                      "max_abs_spread_radius_difference": float(np.max(np.abs(dr))),
                      "spread_radius_difference_at_end": float(dr[-1]),
                      "liquid_regions": {k: {int(st): sn["liquid_regions"] for st, sn in res[k]["snapshots"].items()}
                                         for k in ("original", "corrected")},
                      "contour_segments": {k: {int(st): int(len(sn["contour"])) for st, sn in res[k]["snapshots"].items()}
                                           for k in ("original", "corrected")}}
    return res


def _jsonable(res):
    """The results without field arrays; contours stay, as lists of segments."""
    out = {}
    for k, v in res.items():
        if isinstance(v, dict):
            o = {kk: vv for kk, vv in v.items() if kk != "snapshots"}
            if "snapshots" in v:
                o["contours"] = {int(st): sn["contour"].round(3).tolist() for st, sn in v["snapshots"].items()}
            out[k] = o
        else:
            out[k] = v
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="")
    ap.add_argument("--falling-steps", type=int, default=19000)
    ap.add_argument("--splash-steps", type=int, default=3000)
    args = ap.parse_args()
    res = {"falling_drop": falling_drop(args.falling_steps, direct_defect=True),
           "splash_Re48": splash(48.0, args.splash_steps),
           "splash_Re480": splash(480.0, args.splash_steps),
           "falling_drop_forced": falling_drop(args.falling_steps, f_form=1),
           "splash_Re48_forced": splash(48.0, args.splash_steps, f_form=1),
           "splash_Re480_forced": splash(480.0, args.splash_steps, f_form=1)}
    js = {k: _jsonable(v) for k, v in res.items()}
    text = json.dumps({k: v.get("summary") for k, v in js.items()}, indent=1)
    print(text)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(js, f)


if __name__ == "__main__":
    main()
