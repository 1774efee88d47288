"""Host logic of the closed-surface entry points (include/mbo_surface.h), on
the CPU: the band width, the heat-kernel modes and the sphere and peanut bands
that the library computes on the host (Algorithm 2, step 1) agree with the
oracle, and bad arguments are rejected before any device call."""
import math

import numpy as np
import pytest

from oracle import surface as S
from paper_1711_01365_gb300 import build as B
from paper_1711_01365_gb300 import mbo as M


@pytest.fixture(scope="module")
def lib():
    B.build()
    return M.lib()


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9, 1e-12])
@pytest.mark.parametrize("tau", [1e-1, 1e-2, 5e-3, 1e-4])
def test_band_width_and_modes_match_the_oracle(lib, eps, tau):
    assert M.mbo_surface_band_width(eps, tau) == pytest.approx(S.band_width(eps, tau), rel=1e-12)
    for R in (math.pi, 3.3, 7.0):
        h, m = M.mbo_surface_heat_modes(eps, tau, R)
        ho, mo = S.heat_modes(eps, tau, R)
        assert h == pytest.approx(ho, rel=1e-14)
        assert m == mo


@pytest.mark.parametrize("radius,dx,wb,p", [(1.0, 0.25, 0.4, 2), (1.0, 0.2, 0.57, 3), (1.5, 0.3, 0.3, 1)])
def test_sphere_band_matches_the_oracle(lib, radius, dx, wb, p):
    xq, wq, xc = M.mbo_surface_sphere_band(radius, dx, wb, p)
    oq, ow, oc = S.sphere_band(radius, dx, wb, p)
    assert xq.shape == oq.shape
    assert np.abs(xq - oq).max() < 1e-13
    assert np.abs(wq - ow).max() < 1e-15
    assert np.abs(xc - oc).max() < 1e-13


def test_bad_arguments_rejected(lib):
    assert M.mbo_surface_band_width(0.0, 0.01) < 0
    assert M.mbo_surface_band_width(1e-6, -1.0) < 0
    with pytest.raises(M.MboError) as ei:
        M.mbo_surface_heat_modes(0.7, 0.01, 1.0)
    assert ei.value.status == 1
    with pytest.raises(M.MboError):
        M.mbo_surface_sphere_band(1.0, 0.0, 0.5, 2)
    with pytest.raises(M.MboError):
        M.mbo_surface_peanut_band(0.3, -1.0, 2)
    pts = np.zeros((4, 3))
    w = np.ones(4)
    for args in [(pts, w, pts, 0, 0.01, 1e-6), (pts, w, pts, 5, 0.01, 1e-6), (pts, w, pts, 2, 0.0, 1e-6),
                 (pts, w, pts, 2, 0.01, 0.0), (pts, w, pts, 2, 0.01, 0.7)]:
        with pytest.raises(M.MboError) as ei:
            M.mbo_surface_create(*args)
        assert ei.value.status == 1
    with pytest.raises(M.MboError) as ei:  # no points
        M.mbo_surface_create(np.zeros((0, 3)), np.zeros(0), np.zeros((0, 3)), 2, 0.01, 1e-6)
    assert ei.value.status == 1
    bad = pts.copy()
    bad[1, 2] = np.nan
    with pytest.raises(M.MboError) as ei:
        M.mbo_surface_create(bad, w, pts, 2, 0.01, 1e-6)
    assert ei.value.status == 1


@pytest.mark.parametrize("dx,wb,p", [(0.4, 0.53, 2), (0.35, 1.07, 1), (0.3, 0.77, 2)])
def test_peanut_band_matches_the_oracle(lib, dx, wb, p):
    """Sec. 6.3: the library's peanut band (closest points by its own curve scan
    and golden-section search) against the oracle's.  The search stops at
    ~1e-8 in t, so closest points agree to 1e-6; band widths are chosen away
    from exact ties (a grid point whose distance equals wb)."""
    xq, wq, xc = M.mbo_surface_peanut_band(dx, wb, p)
    oq, ow, oc = S.peanut_band(dx, wb, p)
    assert xq.shape == oq.shape
    assert np.abs(xq - oq).max() < 1e-13
    assert np.abs(wq - ow).max() < 1e-15
    assert np.abs(xc - oc).max() < 1e-6


def test_grid_beyond_2048_rejected(lib):
    """Points 100 apart at tau = 1e-4 need M = 7713 modes per axis (the
    heat-kernel approximation theorem), a grid far beyond 2048 points per
    axis: the plan refuses it before touching the device."""
    h, m = M.mbo_surface_heat_modes(1e-6, 1e-4, 100.0)
    assert 4 * m > 2048
    pts = np.array([[0.0, 0.0, 0.0], [100.0, 100.0, 100.0]])
    with pytest.raises(M.MboError) as ei:
        M.mbo_surface_create(pts, np.ones(2), pts, 2, 1e-4, 1e-6)
    assert ei.value.status == 2
