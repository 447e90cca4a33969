"""Ragged batches: members of different sizes, boundaries and parameters advance in one
persistent launch per step (CUDA-graph replay) and end bitwise where they end alone."""
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


def mix():
    return [
        W.static_droplet(nx=96, ny=64, R=14.0, remove_Fa=1),
        W.random_small(130, 37, seed=3, bc_y=W.WALL, gravity=1e-5),
        W.falling_droplet(nx=64, ny=200, R=12.0, yc=150.0, ratio=10.0, steps=0),
        W.random_small(29, 31, seed=4, bc_x=W.WALL, bc_y=W.WALL, remove_Fa=1),
        W.random_small(300, 70, seed=5, bc_y=W.WALL),
        direct_defect(W.random_small(77, 52, seed=6, bc_y=W.WALL, gravity=1e-5, remove_Fa=1)),
    ]


def direct_defect(w):
    import dataclasses
    return dataclasses.replace(w, phys=dataclasses.replace(w.phys, s_form=1))


def test_alone_equals_in_mix_bitwise(lbm):
    ws = mix()
    alone = []
    for w in ws:
        s = lbm.Sim.from_workload(w)
        s.step(23)
        alone.append(s.moments())
    b = lbm.Batch()
    sims = [lbm.Sim.from_workload(w) for w in ws]
    for s in sims:
        b.add(s)
    b.step(10)
    b.step(13)      # odd count: every member's ping-pong parity flips
    for s, a in zip(sims, alone):
        assert s.step_count == 23
        m = s.moments()
        for k in a:
            assert np.array_equal(m[k], a[k]), k


@pytest.mark.parametrize("plain", [0, 1])
def test_direct_defect_members_in_their_own_launch(lbm, plain):
    """Members with the direct mass defect run in a launch of their own, after the others': with
    and without plain members, in every storage, each member stays bitwise equal to a run alone."""
    base = [W.random_small(77, 52, seed=6, bc_y=W.WALL, gravity=1e-5, remove_Fa=1),
            W.static_droplet(nx=96, ny=64, R=14.0, remove_Fa=1),
            W.random_small(61, 90, seed=9, bc_x=W.WALL, bc_y=W.WALL, remove_Fa=1)]
    members = [(direct_defect(w), st) for w, st in zip(base, (0, 1, 2))]
    if plain:
        members += [(W.random_small(130, 37, seed=3, bc_y=W.WALL, gravity=1e-5), 2),
                    (W.static_droplet(nx=64, ny=64, R=12.0), 0)]
    alone = []
    for w, st in members:
        s = lbm.Sim.from_workload(w, storage=st)
        s.step(17)
        alone.append(s.moments())
    b = lbm.Batch()
    sims = [lbm.Sim.from_workload(w, storage=st) for w, st in members]
    for s in sims:
        b.add(s)
    b.step(6)
    b.step(11)
    for s, a in zip(sims, alone):
        m = s.moments()
        for k in a:
            assert np.array_equal(m[k], a[k]), k


def test_batch_matches_oracle(lbm):
    w = W.random_small(70, 45, seed=8, bc_y=W.WALL, gravity=1e-5, remove_Fa=1)
    b = lbm.Batch()
    s = lbm.Sim.from_workload(w)
    b.add(s)
    b.add(lbm.Sim.from_workload(W.static_droplet(nx=64, ny=64, R=12.0)))
    for _ in range(5):
        b.step(20)
    got = s.moments()
    ref = oracle.run(w, steps=100).moments()
    for k in ("phi", "ux", "uy", "p"):
        den = max(np.abs(ref[k]).max(), 1e-3 if k in ("ux", "uy") else 0.0)
        assert np.abs(got[k] - ref[k]).max() / den < 1e-5, k


def test_membership_changes_and_budget(lbm):
    ws = mix()[:3]
    need = [lbm.device_bytes(w.nx, w.ny) for w in ws]
    b = lbm.Batch(budget_bytes=need[0] + need[1] + need[2] - 1)   # all three never fit together
    sims = [lbm.Sim.from_workload(w) for w in ws]
    s0 = b.add(sims[0])
    b.add(sims[1])
    assert b.try_add(sims[2]) is None            # over budget: refused, nothing allocated
    assert b.size == 2 and b.bytes == need[0] + need[1]
    b.step(7)
    b.remove(s0)                                 # frees budget for the third member
    assert b.try_add(sims[2]) is not None
    b.step(5)
    assert sims[0].step_count == 7 and sims[1].step_count == 12 and sims[2].step_count == 5
    # a removed member steps alone again and its history matches a single run
    sims[0].step(5)
    ref = lbm.Sim.from_workload(ws[0])
    ref.step(12)
    assert np.array_equal(sims[0].moments()["phi"], ref.moments()["phi"])
    with pytest.raises(lbm.LBMError):
        sims[1].step(1)                          # members step only through their batch
