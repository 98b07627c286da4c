"""Diagnostics on the GPU (mmvm_vorticity, mmvm_nonaxi_enstrophy) against the
oracle (oracle/diagnostics.py) and the closed form of the quadrupole's
nonaxisymmetric enstrophy.

Both sides evaluate the same finite sums in FP64 with Hermite polynomials
(recurrence on the GPU, numpy's Hermite series in the oracle): 1e-12 of the
largest |omega| for the vorticity, 1e-10 relative for E (quadrature on the
same polar grid: Gauss-Legendre in r, the trapezoid rule in theta).
"""
import math

import numpy as np
import pytest

import mmvm_inputs
from oracle.coefficients import idx, n_moments
from oracle.diagnostics import nonaxi_enstrophy, vorticity
from oracle.rhs import lam_at

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mm():
    import paper_1010_2475_gb300 as mm

    mm.load_library()
    return mm


@pytest.mark.parametrize("order,n", [(0, 7), (3, 20), (6, 40), (8, 33)])
def test_vorticity_matches_oracle(mm, order, n):
    wl = mmvm_inputs.random_disk(n=n, order=order, radius=2.0, sigma=0.5, amp=0.05,
                                 moment_scale="absolute", seed=70 + order)
    t = 0.6
    pts = np.random.default_rng(order).uniform(-4.0, 4.0, size=(517, 2))
    with mm.Context(order, wl.lam0, wl.nu, mm.MMVM_FP64) as ctx:
        ctx.set_state(wl.x, wl.moments, t)
        g = ctx.vorticity(pts)
    o = vorticity(wl.x, wl.moments, lam_at(t, wl.lam0, wl.nu), order, pts)
    assert np.abs(g - o).max() <= 1e-12 * np.abs(o).max()


def test_vorticity_single_particle_order_20(mm):
    wl = mmvm_inputs.random_disk(n=1, order=20, radius=0.0, sigma=1.0, amp=0.05, seed=5)
    pts = np.random.default_rng(2).uniform(-6.0, 6.0, size=(300, 2))
    with mm.Context(20, wl.lam0, wl.nu, mm.MMVM_FP64) as ctx:
        ctx.set_state(wl.x, wl.moments, 0.0)
        g = ctx.vorticity(pts)
    o = vorticity(wl.x, wl.moments, wl.lam0, 20, pts)
    assert np.abs(g - o).max() <= 1e-12 * np.abs(o).max()


@pytest.mark.parametrize("a,b,lam", [(0.1, 0.0, 1.0), (0.05, 0.08, 1.3)])
def test_quadrupole_enstrophy(mm, a, b, lam):
    order = 4
    mom = np.zeros((1, n_moments(order)))
    mom[0, 0] = 1.0
    mom[0, idx(2, 0)] = a
    mom[0, idx(0, 2)] = -a
    mom[0, idx(1, 1)] = b
    with mm.Context(order, lam, 1e-3, mm.MMVM_FP64) as ctx:
        ctx.set_state(np.zeros((1, 2)), mom, 0.0)
        E = ctx.nonaxi_enstrophy(0.0, 0.0, 10.0 * lam, 64, 64)
    assert E == pytest.approx((4 * a * a + b * b) / (2 * math.pi * lam ** 6), rel=1e-10)


def test_enstrophy_matches_oracle_and_decays(mm):
    """The elliptical Lamb-Oseen perturbation (order 10): E on the GPU equals
    the oracle's on the same grid, and the nonaxisymmetric part decays as the
    vortex axisymmetrises."""
    wl = mmvm_inputs.single_quadrupole(order=10, eps=0.1, sigma0=1.0, Re=1000.0, dt=0.01)
    with mm.Context(10, wl.lam0, wl.nu, mm.MMVM_FP64) as ctx:
        ctx.set_state(wl.x, wl.moments, 0.0)
        E0 = ctx.nonaxi_enstrophy(0.0, 0.0, 9.0, 96, 128)
        ref = nonaxi_enstrophy(wl.x, wl.moments, wl.lam0, 10, r_max=9.0, nr=96, ntheta=128)
        assert E0 == pytest.approx(ref, rel=1e-10)
        ctx.step(wl.dt, 300)
        E1 = ctx.nonaxi_enstrophy(0.0, 0.0, 9.0, 96, 128)
    assert 0.0 < E1 < E0
