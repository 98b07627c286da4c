"""Pins of the oracle on the two-vortex merger model (Section 3.2.1).

Two equal Gaussian vortices at (+-1, 0) (b = 2), circulation 1, nu = 1e-3,
core a; time in turnover units t* = t / (2 pi^2 b^2), up to t* = 0.152.
What the paper's text fixes (its figures print no values):
* m = 0 (pure Gaussians) keeps each centroid at distance 1 from the origin
  for all time (two equal vortices rotate on a circle);
* in the merger regime (a/b = 0.375) the distance falls quickly once
  moments are included, and the trajectory settles as m grows; the text
  quotes a 20 % decline by t* = 0.152 (with lambda_0 = a this oracle gives
  14 %; the test accepts 10-30 %);
* well separated (a/b = 0.125) the distance is kept or falls only slightly.
"""
import math

import numpy as np
import pytest

import mmvm_inputs
from oracle.integrate import dopri5

T_STAR = (0.05, 0.1, 0.127, 0.152)


def radii(a_over_b, order):
    wl = mmvm_inputs.vortex_pair(order=order, a_over_b=a_over_b)
    b = wl.meta["b"]
    x, mom, t = wl.x, wl.moments, 0.0
    out = []
    for ts in T_STAR:
        x, mom, t, _, _ = dopri5(x, mom, t, ts * 2 * math.pi ** 2 * b ** 2, 0.01, order,
                                 wl.lam0, wl.nu, rtol=1e-8, atol=1e-8)
        out.append((np.linalg.norm(x[0]), np.linalg.norm(x[1])))
    return np.array(out)


@pytest.mark.parametrize("a_over_b", [0.375, 0.125])
def test_gaussians_rotate_on_the_circle(a_over_b):
    r = radii(a_over_b, 0)
    assert np.abs(r - 1.0).max() < 1e-9


def test_merger_regime_converges_in_m():
    r = {m: radii(0.375, m) for m in (2, 4, 5, 6)}
    for m in r:
        assert np.abs(r[m][:, 0] - r[m][:, 1]).max() < 1e-9  # the pair stays symmetric
        assert np.all(np.diff(r[m][:, 0]) < 0)  # falls monotonically
    decline = 1.0 - r[6][-1, 0]
    assert 0.10 < decline < 0.30
    assert np.abs(r[6][:, 0] - r[5][:, 0]).max() < 2e-3
    assert np.abs(r[6][:, 0] - r[4][:, 0]).max() < 5e-3
    assert np.abs(r[6][:, 0] - r[2][:, 0]).max() > 0.02  # m = 2 is not yet settled


def test_well_separated_pair_keeps_its_distance():
    for m in (2, 4, 6):
        r = radii(0.125, m)
        assert np.abs(r - 1.0).max() < 0.01
