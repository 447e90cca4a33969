"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded inputs.

Error metric: relative L-infinity, max|gpu - ref| / max|ref|; for the velocity the denominator
is at least the capillary velocity sigma / (rho_A nu_A) (a static droplet's velocity is a
spurious current far below any physical scale).  FP32 tolerance: 1e-5 on phi, u and p.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_5004_gb300 import build
    build.build()
    import paper_1110_5004_gb300 as m
    return m


def rel_errors(got, ref, w):
    u_cap = w.phys.sigma / (w.phys.rho_A * w.phys.nu_A)
    out = {}
    for k in ("phi", "rho", "ux", "uy", "p"):
        den = np.abs(ref[k]).max()
        if k in ("ux", "uy"):
            den = max(np.abs(ref["ux"]).max(), np.abs(ref["uy"]).max(), u_cap)
        den = max(den, 1e-30)
        out[k] = float(np.abs(got[k].astype(np.float64) - ref[k]).max() / den)
    return out


def assert_parity(got, ref, w, tol=TOL):
    err = rel_errors(got, ref, w)
    bad = {k: v for k, v in err.items() if not v <= tol}
    assert not bad, "rel L-inf above %g: %r (all %r)" % (tol, bad, err)
    return err


def run_both(lbm, w, steps, tile=None):
    sim = lbm.Sim.from_workload(w, tile=tile)
    sim.step(steps)
    got = sim.moments()
    ref = oracle.run(w, steps=steps).moments()
    return sim, got, ref


CASES = [
    # nx, ny, bc_x, bc_y, remove_Fa, gravity, seed
    (24, 20, W.PERIODIC, W.PERIODIC, 0, 0.0, 1),
    (24, 20, W.PERIODIC, W.PERIODIC, 1, 0.0, 1),
    (33, 17, W.PERIODIC, W.WALL, 0, 1e-5, 2),
    (33, 17, W.PERIODIC, W.WALL, 1, 1e-5, 2),
    (29, 31, W.WALL, W.WALL, 1, 2e-5, 3),
    (7, 5, W.PERIODIC, W.PERIODIC, 1, 0.0, 4),
    (130, 9, W.WALL, W.PERIODIC, 0, 0.0, 5),
]


@pytest.mark.parametrize("nx,ny,bcx,bcy,rf,g,seed", CASES)
def test_small_grids_200_steps(lbm, nx, ny, bcx, bcy, rf, g, seed):
    w = W.random_small(nx, ny, seed=seed, bc_x=bcx, bc_y=bcy, remove_Fa=rf, gravity=g)
    _, got, ref = run_both(lbm, w, 200)
    assert_parity(got, ref, w)


@pytest.mark.parametrize("bcy", [W.PERIODIC, W.WALL])
def test_conservative_cahn_hilliard_form(lbm, bcy):
    """ch_conservative = 1 (no phi div(u) source) against the oracle in the same form."""
    import dataclasses
    w = W.random_small(61, 37, seed=17, bc_y=bcy, gravity=1e-5 if bcy == W.WALL else 0.0, remove_Fa=1)
    w = dataclasses.replace(w, phys=dataclasses.replace(w.phys, ch_conservative=1))
    _, got, ref = run_both(lbm, w, 200)
    assert_parity(got, ref, w)


@pytest.mark.parametrize("bcy", [W.PERIODIC, W.WALL])
def test_surface_force_mu_grad_phi(lbm, bcy):
    """fs_form = 1 (F_s = mu grad phi) against the oracle in the same form."""
    import dataclasses
    w = W.random_small(58, 41, seed=19, bc_y=bcy, gravity=1e-5 if bcy == W.WALL else 0.0, remove_Fa=1)
    w = dataclasses.replace(w, phys=dataclasses.replace(w.phys, fs_form=1))
    _, got, ref = run_both(lbm, w, 200)
    assert_parity(got, ref, w)


@pytest.mark.parametrize("bcx,bcy", [(W.PERIODIC, W.PERIODIC), (W.PERIODIC, W.WALL), (W.WALL, W.WALL)])
def test_direct_mass_defect(lbm, bcx, bcy):
    """s_form = 1 (mass defect from the stored rho and div(rho u) of the previous step) with
    the corrected scheme, against the oracle in the same form; several tiles and segments."""
    import dataclasses
    w = W.random_small(97, 43, seed=23, bc_x=bcx, bc_y=bcy, gravity=1e-5 if bcy == W.WALL else 0.0, remove_Fa=1)
    w = dataclasses.replace(w, phys=dataclasses.replace(w.phys, s_form=1))
    _, got, ref = run_both(lbm, w, 200, tile=(64, 9))
    assert_parity(got, ref, w)


@pytest.mark.parametrize("bcx,bcy,ch,rf,sform", [
    (W.PERIODIC, W.PERIODIC, 0, 0, 0), (W.PERIODIC, W.WALL, 0, 1, 0), (W.WALL, W.WALL, 1, 1, 0),
    (W.PERIODIC, W.WALL, 0, 1, 1), (W.WALL, W.PERIODIC, 1, 0, 0)])
def test_forced_order_parameter_form(lbm, bcx, bcy, ch, rf, sform):
    """f_form = 1 (forced order-parameter LBE) against the oracle in the same form: periodic and
    walled boxes, both Cahn-Hilliard forms, F_a kept and removed, both mass-defect forms."""
    import dataclasses
    w = W.random_small(71, 39, seed=31 + ch + 2 * rf, bc_x=bcx, bc_y=bcy, gravity=1e-5 if bcy == W.WALL else 0.0,
                       remove_Fa=rf)
    w = dataclasses.replace(w, phys=dataclasses.replace(w.phys, f_form=1, ch_conservative=ch, s_form=sform))
    _, got, ref = run_both(lbm, w, 200, tile=(64, 9))
    assert_parity(got, ref, w)


def test_forced_form_tiles_and_batch(lbm):
    """The forced form's results do not depend on the tile shape (bitwise), and a forced
    simulation cannot join a batch."""
    import dataclasses
    w = W.random_small(130, 44, seed=37, bc_y=W.WALL, gravity=1e-5, remove_Fa=1)
    w = dataclasses.replace(w, phys=dataclasses.replace(w.phys, f_form=1))
    outs = []
    for tile in ((64, 5), (128, 16), (256, 44)):
        s = lbm.Sim.from_workload(w, tile=tile)
        s.step(25)
        outs.append(s.moments())
    for o in outs[1:]:
        for k in o:
            assert np.array_equal(o[k], outs[0][k]), k
    b = lbm.Batch()
    with pytest.raises(Exception):
        b.add(lbm.Sim.from_workload(w))
    b.close()


@pytest.mark.parametrize("rf,sform,bcy", [(0, 0, W.WALL), (1, 0, W.PERIODIC), (0, 1, W.WALL), (1, 1, W.PERIODIC)])
def test_interfacial_force_field(lbm, rf, sform, bcy):
    """F_a = -u s (Eq. 12) of the GPU state against the oracle's, with F_a kept and removed and
    with both mass-defect forms.  Bound: 1e-3 of max|F_a| for the FP32 stencils (s is a second
    difference of mu, itself one of phi), plus, for the direct form, max|u| times 8 ulps of
    rho_A: its rho^t - rho^{t-1} cancels down to the FP32 rounding of the stored densities."""
    import dataclasses
    w = W.random_small(67, 41, seed=27, bc_y=bcy, gravity=1e-5 if bcy == W.WALL else 0.0, remove_Fa=rf)
    w = dataclasses.replace(w, phys=dataclasses.replace(w.phys, s_form=sform))
    sim = lbm.Sim.from_workload(w, tile=(64, 9))
    sim.step(100)
    got, m = sim.interfacial_force(), sim.moments()
    o = oracle.run(w, steps=100)
    ref = {"fax": o.field(oracle.FAX), "fay": o.field(oracle.FAY)}
    umax = float(np.max(np.hypot(m["ux"], m["uy"])))
    for k in ("fax", "fay"):
        scale = float(np.abs(ref[k]).max())
        assert scale > 0.0
        bound = 1e-3 * scale + (umax * 8 * 2.0 ** -24 * w.phys.rho_A if sform else 0.0)
        err = float(np.abs(got[k] - ref[k]).max())
        assert err <= bound, (k, err, bound, scale)


def test_initial_state_moments(lbm):
    """t = 0: the moments of the initial populations (init kernel) match the oracle's."""
    w = W.random_small(45, 38, seed=9, bc_y=W.WALL, gravity=1e-5, remove_Fa=1)
    _, got, ref = run_both(lbm, w, 0)
    assert_parity(got, ref, w)


@pytest.mark.parametrize("tile", [(64, 1), (64, 7), (128, 16), (256, 64), (128, 1000)])
def test_many_tiles_and_ragged_tails(lbm, tile):
    """A grid spanning several strips and segments with ragged last tiles (walls and gravity)."""
    w = W.random_small(300, 70, seed=12, bc_y=W.WALL, gravity=1e-5, remove_Fa=1)
    _, got, ref = run_both(lbm, w, 60, tile=tile)
    assert_parity(got, ref, w)


@pytest.mark.parametrize("nx", [150, 151])
def test_tile_shape_does_not_change_results(lbm, nx):
    """Per-cell arithmetic is independent of the tile shape: bitwise-identical states."""
    w = W.random_small(nx, 44, seed=21, bc_y=W.WALL, gravity=1e-5, remove_Fa=1)
    outs = []
    for tile in ((64, 5), (128, 16), (256, 64), (128, 44)):
        s = lbm.Sim.from_workload(w, tile=tile)
        s.step(37)
        outs.append(s.moments())
    for o in outs[1:]:
        for k in o:
            assert np.array_equal(o[k], outs[0][k]), k


@pytest.mark.parametrize("bcx", [W.PERIODIC, W.WALL])
def test_top_wall_row_inside_segment_fill(lbm, bcx):
    """Segments whose fifth row (first row + 4) is the top wall row: the wall's mirrored ghost
    row shares a ring slot with the segment's first halo row.  On a 29-row walled grid, segment
    heights 8 and 4 both start a segment at row 24; the results must equal the single-segment
    run bitwise and the oracle within tolerance."""
    w = W.random_small(75, 29, seed=41, bc_x=bcx, bc_y=W.WALL, gravity=1e-5, remove_Fa=1)
    outs = []
    for tile in ((64, 29), (64, 8), (128, 4), (64, 1)):
        s = lbm.Sim.from_workload(w, tile=tile)
        s.step(30)
        outs.append(s.moments())
    for o in outs[1:]:
        for k in o:
            assert np.array_equal(o[k], outs[0][k]), k
    assert_parity(outs[0], oracle.run(w, steps=30).moments(), w)


def test_grid_taller_than_a_launch_dimension(lbm):
    """70 000 rows, more than a grid's y dimension allows (65 535): initialisation, steps,
    moments and the FP64 diagnostics against the oracle."""
    w = W.random_small(24, 70000, seed=44, bc_y=W.WALL, gravity=1e-5, remove_Fa=1)
    sim, got, ref = run_both(lbm, w, 3)
    assert_parity(got, ref, w)
    d = sim.diagnostics()
    assert d["finite"] and abs(d["sum_phi"] - float(ref["phi"].sum())) <= 1e-6 * w.cells


@pytest.mark.parametrize("tile", [None, (128, 82)])
def test_largest_serving_request(lbm, tile):
    """The largest grid a c5 request draws (1024 x 4096, falling drop between walls, corrected
    scheme), at full size against the oracle over 5 steps, with the default tile and the
    whole-wave tile the tuner offers there (9 strips x 50 segments of 82 rows, 3 CTAs per SM)."""
    w = W.falling_droplet(nx=1024, ny=4096, R=120.0, yc=3400.0, ratio=10.0, remove_Fa=1)
    _, got, ref = run_both(lbm, w, 5, tile=tile)
    assert_parity(got, ref, w)


def test_large_periodic_grid_on_the_tuned_tile(lbm):
    """The 4096 x 4096 periodic static drop of the benchmark's large-grid line (2.4 GB of
    populations, far beyond L2), at full size against the oracle over 3 steps on the tile the
    tuner picks on GB300 (128 threads x 316 rows: 34 strips x 13 segments)."""
    w = W.static_droplet(nx=4096, ny=4096, R=600.0)
    _, got, ref = run_both(lbm, w, 3, tile=(128, 316))
    assert_parity(got, ref, w)


@pytest.mark.parametrize("nx,tile", [(3193, (64, 0)), (14521, (128, 0)), (131, (64, 9)), (250, (64, 9))])
def test_strip_ending_short_of_a_side_wall(lbm, nx, tile):
    """Side walls with many strips, among them the widths whose second-to-last strip ends 3
    columns before the right wall (64 threads: 58-column strips; 128 threads: 122-column
    strips), so the wall's ghost column falls just outside that strip's ring."""
    w = W.random_small(nx, 6, seed=30 + nx % 7, bc_x=W.WALL, bc_y=W.WALL, gravity=1e-5, remove_Fa=1)
    _, got, ref = run_both(lbm, w, 20, tile=tile)
    assert_parity(got, ref, w)


TILE_CASES = [
    # nx, ny, bc_x, bc_y, remove_Fa, ch_conservative, fs_form, storage, seed
    (24, 20, W.PERIODIC, W.PERIODIC, 0, 0, 0, 0, 1),
    (33, 17, W.PERIODIC, W.WALL, 1, 0, 0, 0, 2),
    (29, 31, W.WALL, W.WALL, 1, 0, 1, 0, 3),
    (7, 5, W.PERIODIC, W.PERIODIC, 1, 1, 0, 0, 4),
    (130, 9, W.WALL, W.PERIODIC, 0, 1, 1, 0, 5),
    (47, 38, W.WALL, W.WALL, 1, 0, 0, 1, 6),
    (40, 24, W.PERIODIC, W.WALL, 0, 0, 0, 2, 7),
    (150, 90, W.PERIODIC, W.WALL, 1, 0, 0, 0, 8),
    # more tiles than one wave of the 384-thread form: the 256-thread form runs
    (400, 200, W.WALL, W.PERIODIC, 1, 1, 0, 0, 12),
    (400, 200, W.PERIODIC, W.WALL, 0, 0, 1, 1, 13),
]


@pytest.mark.parametrize("nx,ny,bcx,bcy,rf,ch,fs,st,seed", TILE_CASES)
def test_tile_kernel_equals_row_march(lbm, nx, ny, bcx, bcy, rf, ch, fs, st, seed):
    """The small-grid tile kernel computes every cell bitwise as the row march: the whole state
    after 40 steps on odd and ragged grids (edge tiles cut by the grid), walls on either axis,
    both schemes, both Cahn-Hilliard forms, both surface forces and every storage."""
    import dataclasses
    w = W.random_small(nx, ny, seed=seed, bc_x=bcx, bc_y=bcy, gravity=1e-5 if bcy == W.WALL else 0.0,
                       remove_Fa=rf)
    w = dataclasses.replace(w, phys=dataclasses.replace(w.phys, ch_conservative=ch, fs_form=fs))
    rows = lbm.Sim.from_workload(w, storage=st, kernel=lbm.LBM_KERNEL_ROWS)
    tiles = lbm.Sim.from_workload(w, storage=st, kernel=lbm.LBM_KERNEL_TILES)
    rows.step(40)
    tiles.step(40)
    assert np.array_equal(tiles.checkpoint(), rows.checkpoint())


RESIDENT_CASES = TILE_CASES + [
    # more tiles than one wave of resident CTAs: each CTA steps several tiles in turn
    (300, 150, W.PERIODIC, W.WALL, 1, 0, 0, 0, 9),
    (512, 512, W.PERIODIC, W.PERIODIC, 0, 0, 0, 0, 10),
    (250, 300, W.WALL, W.WALL, 0, 1, 0, 1, 11),
]


@pytest.mark.parametrize("nx,ny,bcx,bcy,rf,ch,fs,st,seed", RESIDENT_CASES)
def test_resident_kernel_equals_tile_kernel(lbm, nx, ny, bcx, bcy, rf, ch, fs, st, seed):
    """The resident form (n steps in one launch, each tile waiting only on the tiles within its
    reach) gives the tile kernel's state bitwise, over several calls of odd and even lengths (a
    launch that starts from either buffer, the flags carried from one launch to the next)."""
    import dataclasses
    w = W.random_small(nx, ny, seed=seed, bc_x=bcx, bc_y=bcy, gravity=1e-5 if bcy == W.WALL else 0.0,
                       remove_Fa=rf)
    w = dataclasses.replace(w, phys=dataclasses.replace(w.phys, ch_conservative=ch, fs_form=fs))
    tiles = lbm.Sim.from_workload(w, storage=st, kernel=lbm.LBM_KERNEL_TILES)
    res = lbm.Sim.from_workload(w, storage=st, kernel=lbm.LBM_KERNEL_RESIDENT)
    for n in (7, 1, 12, 20):
        tiles.step(n)
        before = res.launch_count
        res.step(n)
        assert res.launch_count - before == 1
        assert res.step_status() == 0
        assert np.array_equal(res.checkpoint(), tiles.checkpoint()), n


def test_resident_wait_runs_out_and_recovers(lbm):
    """A tile that never announces its step (the host's hold_tile hook) makes its neighbours'
    bounded waits run out: the launch ends by itself well within a second, lbm_step_status and
    lbm_diagnostics report LBM_ERR_TIMEOUT, later launches do nothing until the status is read,
    and after a new initial state the resident kernel again matches the tile kernel bitwise."""
    import time
    w = W.static_droplet()
    res = lbm.Sim.from_workload(w, kernel=lbm.LBM_KERNEL_RESIDENT)
    res.set_wait_limit(20_000_000, hold_tile=37)         # 20 ms
    t0 = time.perf_counter()
    res.step(50)
    assert res.step_status() == lbm._lib.LBM_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert res.step_status() == 0                        # read once, then re-armed
    res.step(10)                                         # held again: gives up again
    with pytest.raises(lbm.LBMError) as e:
        res.diagnostics()
    assert e.value.code == lbm._lib.LBM_ERR_TIMEOUT
    res.set_wait_limit(1_000_000_000)                    # no tile held
    res.init_fields(*[np.ascontiguousarray(a, np.float32) for a in (w.phi0, w.ux0, w.uy0, w.p0)])
    tiles = lbm.Sim.from_workload(w, kernel=lbm.LBM_KERNEL_TILES)
    res.step(30)
    tiles.step(30)
    assert res.step_status() == 0
    assert np.array_equal(res.checkpoint(), tiles.checkpoint())
    assert res.diagnostics()["finite"]


def test_active_kernel_follows_the_measured_crossover(lbm):
    """AUTO runs the tile kernel on grids of up to 262144 cells (where it was measured faster,
    with and without x walls), the row march above, and the row march wherever the tile kernel
    does not apply; an explicit choice is reported as made."""
    import dataclasses
    xwall = lambda w: dataclasses.replace(w, phys=dataclasses.replace(w.phys, bc_x=W.WALL))
    cases = [(W.static_droplet(), lbm.LBM_KERNEL_TILES),
             (W.static_droplet(nx=512, ny=512, R=100), lbm.LBM_KERNEL_TILES),    # 262144 cells
             (W.falling_droplet(), lbm.LBM_KERNEL_TILES),
             (xwall(W.static_droplet(nx=512, ny=512, R=100)), lbm.LBM_KERNEL_TILES),
             (W.static_droplet(nx=513, ny=512, R=100), lbm.LBM_KERNEL_ROWS),
             (xwall(W.static_droplet(nx=1024, ny=512, R=100)), lbm.LBM_KERNEL_ROWS)]
    for w, want in cases:
        s = lbm.Sim.from_workload(w, init=False)
        assert s.active_kernel == want, (w.nx, w.ny)
        s.close()
    w = W.random_small(40, 24, seed=3)
    s = lbm.Sim.from_workload(w, init=False, kernel=lbm.LBM_KERNEL_RESIDENT)
    assert s.active_kernel == lbm.LBM_KERNEL_RESIDENT
    s.set_kernel(lbm.LBM_KERNEL_ROWS)
    assert s.active_kernel == lbm.LBM_KERNEL_ROWS
    s.close()
    w = dataclasses.replace(w, phys=dataclasses.replace(w.phys, s_form=1))
    s = lbm.Sim.from_workload(w, init=False)
    assert s.active_kernel == lbm.LBM_KERNEL_ROWS
    s.close()


def test_tile_kernel_refused_where_it_does_not_apply(lbm):
    import dataclasses
    w = W.random_small(40, 24, seed=3)
    w = dataclasses.replace(w, phys=dataclasses.replace(w.phys, s_form=1))
    s = lbm.Sim.from_workload(w)
    with pytest.raises(lbm.LBMError):
        s.set_kernel(lbm.LBM_KERNEL_TILES)
    with pytest.raises(lbm.LBMError):
        s.set_kernel(lbm.LBM_KERNEL_RESIDENT)


@pytest.mark.parametrize("rf", [0, 1])
def test_c1_static_droplet(lbm, rf):
    """c1 (128x128 periodic, R = 25, rho 1:0.1): 1e-5 after 200 steps; the full 1000-step run
    stays within tolerance too."""
    w = W.static_droplet(remove_Fa=rf)
    sim = lbm.Sim.from_workload(w)
    ref = oracle.Sim.from_workload(w)
    sim.step(200)
    ref.step(200)
    assert_parity(sim.moments(), ref.moments(), w)
    sim.step(800)
    ref.step(800)
    assert_parity(sim.moments(), ref.moments(), w)
    dg, dr = sim.diagnostics(), ref.diagnostics()
    assert dg["step"] == dr["step"] == 1000
    assert dg["sum_phi"] == pytest.approx(dr["sum_phi"], rel=1e-6)
    assert dg["centroid_x"] == pytest.approx(dr["centroid_x"], rel=1e-6)
    assert dg["spread_radius"] == pytest.approx(dr["spread_radius"], rel=1e-5)
    assert dg["p_liquid"] == pytest.approx(dr["p_liquid"], rel=1e-5)


def test_c2_falling_droplet_until_divergence(lbm):
    """c2 (256x1024, walls, rho 1:0.01): 1e-5 at steps 30 and 100 (measured 1.5e-6 and
    3.6e-6; the gap grows only as the run nears its divergence, after step 125); both sides
    diverge (the central-difference scheme's density-ratio limit) at the same step."""
    w = W.falling_droplet()
    sim = lbm.Sim.from_workload(w)
    ref = oracle.Sim.from_workload(w)
    sim.step(30)
    ref.step(30)
    assert_parity(sim.moments(), ref.moments(), w)
    sim.step(70)
    ref.step(70)
    assert_parity(sim.moments(), ref.moments(), w)
    first = {}
    for k in range(100, 600):
        for name, s in (("gpu", sim), ("ref", ref)):
            if name not in first and not s.diagnostics()["finite"]:
                first[name] = k
        if len(first) == 2:
            break
        sim.step(1)
        ref.step(1)
    assert "gpu" in first and "ref" in first
    assert abs(first["gpu"] - first["ref"]) <= 2


@pytest.mark.parametrize("tile", [None, (128, 15), (128, 20), (256, 16)])
def test_c3_splash_until_divergence(lbm, tile):
    """c3 (2048x512, rho 1:0.001, Re 500, We 8000): 1e-5 after 3 and 5 steps at full size
    (measured 1.5e-6 and 1.6e-6; from step 6 the run's own instability amplifies rounding), with
    the default tile (one wave of CTAs) and with the tiles the benchmark's tuner chooses between
    on GB300 (128 threads x 15 rows: 595 CTAs, 4 per SM; 128 x 20: 3 per SM; 256 x 16); both
    sides diverge within the first dozen steps."""
    w = W.splash()
    sim = lbm.Sim.from_workload(w, tile=tile)
    ref = oracle.Sim.from_workload(w)
    sim.step(3)
    ref.step(3)
    assert_parity(sim.moments(), ref.moments(), w)
    sim.step(2)
    ref.step(2)
    assert_parity(sim.moments(), ref.moments(), w)
    for _ in range(18):
        sim.step(1)
        ref.step(1)
    assert not sim.diagnostics()["finite"] and not ref.diagnostics()["finite"]


def c3_16bit_phi_error(lbm, st, tile):
    w = W.splash()
    sim = lbm.Sim.from_workload(w, tile=tile, storage=st)
    sim.step(3)
    ref = oracle.run(w, steps=3).moments()
    got = sim.moments()
    return float(np.abs(got["phi"] - ref["phi"]).max() / np.abs(ref["phi"]).max())


@pytest.mark.parametrize("tile", [(128, 15), (128, 20), (256, 16)])
def test_c3_splash_fp16_storage(lbm, tile):
    """c3 at full size with FP16 population storage (FP32 arithmetic) on the tiles the
    benchmark's tuner chooses between: phi within the reduced-storage bound of 1e-3 of the FP64
    oracle after 3 steps."""
    err = c3_16bit_phi_error(lbm, 1, tile)
    assert err <= 1e-3, err


@pytest.mark.parametrize("tile", [(128, 20)])
def test_c3_splash_bf16_storage(lbm, tile):
    """c3 at full size with BF16 population storage (stochastic rounding, FP32 arithmetic): phi
    within the reduced-storage bound of 1e-3 of the FP64 oracle after 3 steps (measured 4.2e-4)."""
    err = c3_16bit_phi_error(lbm, 2, tile)
    assert err <= 1e-3, err


@pytest.mark.parametrize("st", [0, 1, 2])
def test_diverged_state_reports_error_code(lbm, st):
    """A state that left the finite range is reported in every storage: 16-bit stores keep NaN
    and infinity non-finite (BF16's stochastic rounding included)."""
    w = W.splash(nx=256, ny=128, D=50)
    sim = lbm.Sim.from_workload(w, storage=st)
    sim.step(30)
    with pytest.raises(lbm.LBMError) as e:
        sim.diagnostics(raise_on_divergence=True)
    assert e.value.code == lbm.LBM_ERR_DIVERGED


def test_diagnostics_match_oracle(lbm):
    w = W.falling_droplet(nx=96, ny=160, R=20.0, yc=100.0, ratio=10.0, steps=0)
    sim = lbm.Sim.from_workload(w)
    ref = oracle.Sim.from_workload(w)
    sim.step(150)
    ref.step(150)
    dg, dr = sim.diagnostics(), ref.diagnostics()
    for k in ("sum_phi", "liquid_area", "centroid_x", "centroid_y", "spread_radius", "p_liquid", "p_gas"):
        assert dg[k] == pytest.approx(dr[k], rel=1e-5, abs=1e-9), k
    for k in ("vel_x", "vel_y", "max_u"):
        assert dg[k] == pytest.approx(dr[k], rel=1e-4, abs=1e-9), k
    assert dg["finite"] == 1 and dg["step"] == 150


def test_diagnostics_are_bitwise_reproducible(lbm):
    w = W.random_small(64, 48, seed=2)
    sim = lbm.Sim.from_workload(w)
    sim.step(10)
    a, b = sim.diagnostics(), sim.diagnostics()
    assert a == b


def test_device_pointers_in_and_out(lbm):
    """Fields may be torch CUDA tensors on both sides of the ABI."""
    import torch
    w = W.random_small(40, 24, seed=6, bc_y=W.WALL)
    s = lbm.Sim(w.nx, w.ny, lbm.params_from_physical(w.phys))
    dev = {k: torch.from_numpy(getattr(w, k)).cuda() for k in ("phi0", "ux0", "uy0", "p0")}
    s.init_fields(dev["phi0"], dev["ux0"], dev["uy0"], dev["p0"])
    s.step(25)
    out = {k: torch.empty((w.ny, w.nx), device="cuda") for k in ("phi", "rho", "ux", "uy", "p")}
    s.moments(out)
    host = lbm.Sim.from_workload(w)
    host.step(25)
    h = host.moments()
    for k in out:
        assert np.array_equal(out[k].cpu().numpy(), h[k]), k


def test_pinned_input_consumed_when_phi0_is_on_the_device(lbm):
    """lbm_init_fields returns only once every host input has been copied, whatever phi0 is:
    here phi0, uy0 and p0 are device tensors and ux0 a page-locked host buffer, which the caller overwrites
    right after the call.  The state equals one initialised from pageable copies, bitwise."""
    import torch
    w = W.random_small(96, 40, seed=8, bc_y=W.WALL)
    s = lbm.Sim(w.nx, w.ny, lbm.params_from_physical(w.phys))
    phi_dev, uy_dev, p_dev = (torch.from_numpy(a).cuda() for a in (w.phi0, w.uy0, w.p0))
    torch.cuda.synchronize()
    ux_pin = torch.from_numpy(w.ux0.copy()).pin_memory()
    s.init_fields(phi_dev, ux_pin, uy_dev, p_dev)   # the only host input is pinned
    ux_pin.fill_(float("nan"))   # reused by the caller at once
    s.step(5)
    ref = lbm.Sim.from_workload(w)
    ref.step(5)
    got, want = s.moments(), ref.moments()
    for k in got:
        assert np.array_equal(got[k], want[k]), k


@pytest.mark.parametrize("nx", [64, 40])
def test_moments_into_pinned_host_and_device_buffers(lbm, nx):
    """With nx a multiple of 32 the moment pass writes device tensors itself (no staging copy);
    page-locked host buffers, and every target at other widths, are copied from the pitched work
    planes.  Either way, and with targets of every kind mixed in one call, the fields equal those
    the copy path delivers into pageable arrays, bitwise."""
    import torch
    names = ("phi", "rho", "ux", "uy", "p")
    w = W.random_small(nx, 24, seed=6, bc_y=W.WALL, remove_Fa=1)
    s = lbm.Sim.from_workload(w)
    s.step(25)
    ref = s.moments()                                   # pageable numpy outputs: copied
    nan = float("nan")
    pinned = {k: torch.full((w.ny, w.nx), nan).pin_memory() for k in names}
    dev = {k: torch.full((w.ny, w.nx), nan, device="cuda") for k in names}
    s.moments(pinned)
    s.moments(dev)
    for k in names:
        assert np.array_equal(pinned[k].numpy(), ref[k]), ("pinned", k)
        assert np.array_equal(dev[k].cpu().numpy(), ref[k]), ("device", k)
    mixed = {"phi": torch.full((w.ny, w.nx), nan).pin_memory(), "rho": np.full((w.ny, w.nx), nan, np.float32),
             "ux": torch.full((w.ny, w.nx), nan, device="cuda"), "p": torch.full((w.ny, w.nx), nan).pin_memory()}
    s.moments(mixed)
    for k, v in mixed.items():
        got = v if isinstance(v, np.ndarray) else v.cpu().numpy()
        assert np.array_equal(got, ref[k]), ("mixed", k)


@pytest.mark.parametrize("nx", [64, 45])
def test_packed_fields_in_and_out(lbm, nx):
    """lbm_init_fields_packed / lbm_moments_packed move every field in one block and one copy;
    host and device blocks, rows equal to the work pitch (64) or not (45), give the state and the
    moments of the per-field calls bitwise."""
    import torch
    w = W.random_small(nx, 27, seed=15, bc_y=W.WALL, gravity=1e-5, remove_Fa=1)
    ref = lbm.Sim.from_workload(w)
    ref.step(9)
    want = ref.moments()
    block = np.stack([w.phi0, w.ux0, w.uy0, w.p0]).astype(np.float32)
    names = ("phi", "rho", "ux", "uy", "p")
    for where in ("host", "device"):
        s = lbm.Sim(w.nx, w.ny, lbm.params_from_physical(w.phys))
        src = block if where == "host" else torch.from_numpy(block).cuda()
        s.init_fields_packed(src)
        s.step(9)
        assert np.array_equal(s.checkpoint(), ref.checkpoint()), where
        out = None if where == "host" else torch.full((5, w.ny, w.nx), float("nan"), device="cuda")
        got = s.moments_packed(out)
        got = got if where == "host" else got.cpu().numpy()
        for k, name in enumerate(names):
            assert np.array_equal(got[k], want[name]), (where, name)


def test_zero_steps_and_null_outputs(lbm):
    w = W.random_small(16, 16, seed=1)
    s = lbm.Sim.from_workload(w)
    s.step(0)
    assert s.step_count == 0
    o = {"phi": np.empty((16, 16), np.float32)}
    s.moments(o)
    assert np.isfinite(o["phi"]).all()


def test_corrected_scheme_with_strong_mass_defect(lbm):
    """An interface twice as sharp as its equilibrium width relaxes by Cahn-Hilliard diffusion,
    so the mass defect s = rho' theta_M lap(mu) reaches ~0.4 % of rho: the corrected scheme's
    (rho - s/2) velocity denominator and the u s force are exercised at full strength, with a
    viscosity contrast between the phases."""
    nx, ny = 48, 40
    phi0 = W.droplet_phi(nx, ny, 24, 20, 10, 3.0)
    phys = W.Physical(sigma=0.02, W=6.0, theta_M=0.3, nu_A=0.05, nu_B=0.3, rho_A=1.0, rho_B=0.2,
                      remove_Fa=1)
    w = W.make("mass_defect", nx, ny, phys, 0, phi0)
    _, got, ref = run_both(lbm, w, 20)
    assert_parity(got, ref, w)
