"""Pins of the oracle's vorticity reconstruction and nonaxisymmetric enstrophy
(oracle/diagnostics.py) to closed forms.

* int omega dx = sum_j M^j_00 (only k = 0 carries circulation, eq:mass).
* int x_1 omega dx = sum_j (M^j_00 x^j_1 - M^j_(1,0)) (integration by parts:
  only k = (0,0) and k = (1,0) see the linear weight).
* The Lamb-Oseen core-mismatch state of Section 4.1.1 reconstructs
  sum_n (d/4)^n / n! Lap^n phi_00 with Lap^n phi_00 = (-4/lambda^2)^n n!
  L_n(r^2/lambda^2) phi_00 (Laguerre polynomials), an independent formula.
* A quadrupole a (phi_20 - phi_02) + b phi_11 about a Gaussian core has
  E = (4 a^2 + b^2) / (2 pi lambda^6): with phi_20 - phi_02 = 4 r^2 cos(2 theta)
  phi_00 / lambda^4 and phi_11 = 2 r^2 sin(2 theta) phi_00 / lambda^4,
  E = pi (16 a^2 + 4 b^2) lambda^-8 int r^5 phi_00^2 dr and that integral is
  lambda^2 / (8 pi^2).
"""
import math

import numpy as np
import pytest
from numpy.polynomial import laguerre

import mmvm_inputs
from oracle.coefficients import idx, n_moments
from oracle.diagnostics import nonaxi_enstrophy, polar_grid, vorticity


def _integrate(x, mom, lam, order, weight=None):
    pts, r, wr, dth = polar_grid(0.0, 0.0, 12.0, 96, 96)
    w = vorticity(x, mom, lam, order, pts)
    if weight is not None:
        w = w * weight(pts)
    return float(np.sum(wr[:, None] * w.reshape(96, 96)) * dth)


@pytest.mark.parametrize("order", [0, 3, 6])
def test_circulation_and_first_moment(order):
    wl = mmvm_inputs.random_disk(n=5, order=order, radius=1.5, sigma=0.6, amp=0.05,
                                 moment_scale="absolute", seed=31 + order)
    mom = wl.moments.copy()
    if order >= 1:
        mom[:, 1:3] = np.random.default_rng(order).normal(size=(5, 2)) * 0.05
    circ = _integrate(wl.x, mom, wl.lam0, order)
    assert circ == pytest.approx(mom[:, 0].sum(), abs=1e-11)
    m1 = _integrate(wl.x, mom, wl.lam0, order, weight=lambda p: p[:, 0])
    expect = np.sum(mom[:, 0] * wl.x[:, 0]) - (mom[:, 1].sum() if order >= 1 else 0.0)
    assert m1 == pytest.approx(expect, abs=1e-11)


def test_lamb_oseen_expansion_matches_laguerre_form():
    order, lam, d = 12, 2.0, 2.1 ** 2 - 2.0 ** 2
    mom = np.zeros((1, n_moments(order)))
    for a in range(order // 2 + 1):
        for b in range(order // 2 + 1 - a):
            mom[0, idx(2 * a, 2 * b)] = (d / 4) ** (a + b) / (math.factorial(a) * math.factorial(b))
    r = np.linspace(0.0, 9.0, 91)
    th = 0.37
    pts = np.stack([r * math.cos(th), r * math.sin(th)], axis=1)
    w = vorticity(np.zeros((1, 2)), mom, lam, order, pts)
    phi00 = np.exp(-r ** 2 / lam ** 2) / (math.pi * lam ** 2)
    ref = np.zeros_like(r)
    for nn in range(order // 2 + 1):
        c = np.zeros(nn + 1)
        c[nn] = 1.0
        lap_n = (-4.0 / lam ** 2) ** nn * math.factorial(nn) * laguerre.lagval(r ** 2 / lam ** 2, c)
        ref += (d / 4) ** nn / math.factorial(nn) * lap_n * phi00
    assert np.abs(w - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("a,b,lam", [(0.1, 0.0, 1.0), (0.05, 0.08, 1.3), (0.0, 0.2, 0.7)])
def test_quadrupole_enstrophy_closed_form(a, b, lam):
    order = 4
    mom = np.zeros((1, n_moments(order)))
    mom[0, 0] = 1.0
    mom[0, idx(2, 0)] = a
    mom[0, idx(0, 2)] = -a
    mom[0, idx(1, 1)] = b
    E = nonaxi_enstrophy(np.zeros((1, 2)), mom, lam, order, r_max=10.0 * lam, nr=64, ntheta=64)
    assert E == pytest.approx((4 * a * a + b * b) / (2 * math.pi * lam ** 6), rel=1e-11)


def test_axisymmetric_state_has_no_nonaxisymmetric_enstrophy():
    order = 8
    mom = np.zeros((1, n_moments(order)))
    for a in range(order // 2 + 1):
        for b in range(order // 2 + 1 - a):
            mom[0, idx(2 * a, 2 * b)] = 0.3 ** (a + b) * math.comb(a + b, a) / math.factorial(a + b)
    E = nonaxi_enstrophy(np.zeros((1, 2)), mom, 1.1, order)
    assert E < 1e-28
