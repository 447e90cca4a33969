"""16-bit population storage (FP16 scaled / BF16, FP32 arithmetic) against the FP64 oracle.

Bounds: relative L-infinity on phi <= 1e-3; total-phi drift and the droplet's centroid velocity
within 0.5 %.  The rest population stays FP32 (see lbm_device.cuh); the 17 other populations are
16-bit, so a run moves 76 B per lattice update instead of 152.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_5004_gb300 import build
    build.build()
    import paper_1110_5004_gb300 as m
    return m


STORAGES = [("fp16", 1), ("bf16", 2)]


def rel_linf(a, b):
    return float(np.abs(a.astype(np.float64) - b).max() / np.abs(b).max())


@pytest.mark.parametrize("name,st", STORAGES)
def test_static_droplet_1000_steps(lbm, name, st):
    w = W.static_droplet()
    sim = lbm.Sim.from_workload(w, storage=st)
    sim.step(1000)
    got = sim.moments()
    ref = oracle.run(w, steps=1000)
    r = ref.moments()
    assert rel_linf(got["phi"], r["phi"]) <= 1e-3
    d0 = float(w.phi0.astype(np.float64).sum())
    drift = abs(sim.diagnostics()["sum_phi"] - d0) / abs(d0)
    assert drift <= 5e-3, drift
    # the pressure jump keeps its sign and size (within 2 %)
    dg, dr = sim.diagnostics(), ref.diagnostics()
    assert (dg["p_liquid"] - dg["p_gas"]) == pytest.approx(dr["p_liquid"] - dr["p_gas"], rel=2e-2)


def falling_drop_errors(lbm, st):
    """A falling droplet (rho 1:0.1, walls on y) for 1500 steps against the FP64 oracle:
    relative centroid-velocity error, relative L-inf on phi, relative total-phi difference."""
    w = W.falling_droplet(nx=96, ny=200, R=16.0, yc=140.0, ratio=10.0, gravity=5e-6, nu_A=0.1,
                          visc_ratio=1.0, steps=0)
    sim = lbm.Sim.from_workload(w, storage=st)
    ref = oracle.Sim.from_workload(w)
    sim.step(1500)
    ref.step(1500)
    dg, dr = sim.diagnostics(), ref.diagnostics()
    assert dr["vel_y"] < -1e-4                         # it does fall
    return (abs(dg["vel_y"] - dr["vel_y"]) / abs(dr["vel_y"]),
            rel_linf(sim.moments()["phi"], ref.moments()["phi"]),
            abs(dg["sum_phi"] - dr["sum_phi"]) / abs(dr["sum_phi"]))


@pytest.mark.parametrize("name,st", STORAGES)
def test_falling_droplet_centroid_velocity(lbm, name, st):
    """The stated reduced-storage bounds: phi within 1e-3, centroid velocity and total phi within
    0.5 %.  BF16 meets them through stochastic rounding; with round-to-nearest it missed them
    (3.6 % off in centroid velocity, 1.0e-2 in phi: its 8-bit significand biased populations that
    change little between steps the same way every step)."""
    vel, phi, mass = falling_drop_errors(lbm, st)
    assert vel <= 5e-3, vel
    assert phi <= 1e-3, phi
    assert mass <= 5e-3, mass


def test_bf16_known_shortfall_stays_as_measured(lbm):
    """BF16's documented shortfall on the falling drop, held where it was measured so that a
    regression shows: centroid velocity within 6 % and phi within 3e-2 of the oracle."""
    vel, phi, mass = falling_drop_errors(lbm, 2)
    assert vel <= 6e-2, vel
    assert phi <= 3e-2, phi
    assert mass <= 5e-3, mass


@pytest.mark.parametrize("name,st", STORAGES)
def test_16bit_alone_equals_in_batch(lbm, name, st):
    w = W.random_small(70, 33, seed=13, bc_y=W.WALL, gravity=1e-5)
    a = lbm.Sim.from_workload(w, storage=st)
    a.step(17)
    b = lbm.Batch()
    s = lbm.Sim.from_workload(w, storage=st)
    b.add(s)
    b.add(lbm.Sim.from_workload(W.static_droplet(nx=64, ny=64, R=12.0)))   # FP32 member in the mix
    b.step(17)
    ma, mb = a.moments(), s.moments()
    for k in ma:
        assert np.array_equal(ma[k], mb[k]), k


def test_device_bytes_of_16bit_storage(lbm):
    fp32 = lbm.device_bytes(256, 100, 0)
    fp16 = lbm.device_bytes(256, 100, 1)
    plane = 100 * 256
    assert fp32 - fp16 == 2 * (19 * 4 - 38) * plane
