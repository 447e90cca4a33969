"""Host-side post-processing of the paper's splash output (CPU only): the rho = 0.55 density
contour by marching squares and the count of liquid regions (the drop, the film and any
secondary droplets of the paper's Fig. 2)."""
import math

import numpy as np
import pytest

from paper_1110_5004_gb300 import experiments as E


def disk_rho(nx, ny, xc, yc, R, W=3.0, rho_l=1.0, rho_g=0.1):
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.hypot(x - xc, y - yc)
    c = 0.5 * (1.0 + np.tanh(2.0 * (R - r) / W))
    return rho_g + c * (rho_l - rho_g)


@pytest.mark.parametrize("R", [8.0, 20.0])
def test_contour_of_a_disk_is_a_circle(R):
    rho = disk_rho(80, 70, 40.3, 33.7, R)
    seg = E.contour_segments(rho, 0.55)
    length = np.linalg.norm(seg[:, 1] - seg[:, 0], axis=1).sum()
    # rho = 0.55 is the mid level of the tanh profile: the circle r = R
    assert length == pytest.approx(2 * math.pi * R, rel=1.5e-2)
    mid = seg.mean(axis=1)
    r = np.hypot(mid[:, 0] - 40.3, mid[:, 1] - 33.7)
    assert np.abs(r - R).max() < 0.15


def test_contour_is_empty_without_a_crossing():
    assert len(E.contour_segments(np.full((10, 12), 0.2), 0.55)) == 0


def test_liquid_regions_counts_drops_film_and_periodic_wrap():
    rho = np.maximum(disk_rho(100, 60, 30, 40, 6), disk_rho(100, 60, 70, 40, 5))
    film = np.zeros((60, 100))
    film[:8] = 1.0
    assert E.liquid_regions(rho) == 2
    assert E.liquid_regions(np.maximum(rho, film)) == 3
    wrap = np.maximum(disk_rho(100, 60, 1.0, 30, 6), disk_rho(100, 60, 101.0, 30, 6))   # a drop across x = 0
    assert E.liquid_regions(wrap, periodic_x=False) == 2
    assert E.liquid_regions(wrap, periodic_x=True) == 1
