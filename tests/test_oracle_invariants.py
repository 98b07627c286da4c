"""Pins of the oracle's RHS and RK4 to what the paper and the mathematics fix.

P-1  An axisymmetric single vortex, M_(2a,2b) = g_{a+b} C(a+b, a) (all other
     moments 0), is omega = sum_n g_n Lap^n phi_00: radial, so u . grad omega
     = 0 and the RHS vanishes identically.
P-2  The paper's convergence test (Section 4.1.1): a Lamb-Oseen vortex of true
     core mu_0 = 2.1 expanded at lambda_0 = 2 has M_(2a,2b) = (d/4)^{a+b}/(a!b!),
     d = mu_0^2 - lambda_0^2 (the heat semigroup exp((d/4) Lap) maps one
     Gaussian to the other), is stationary under the MMVM, and its truncation
     error falls geometrically in M.
P-3  dM^j_00/dt = 0 (total vorticity of each particle, eq:mass).
P-4  dM^j_(1,0)/dt = dM^j_(0,1)/dt = 0 for any state (the centroid condition
     eq:xjdef is what defines xdot^j).
P-5  sum_j M^j_00 xdot^j = 0 (linear impulse).
P-9  M = 0 is the core-spreading vortex method (Section 3.2.2): two vortices
     rotate rigidly with Omega = (G1+G2)/(2 pi d^2) (1 - exp(-d^2/(2 lambda^2))).
P-10 Covariance under a 90-degree rotation and under a reflection.
     RK4 is fourth order (halving dt divides the error by ~16).
"""
import math

import numpy as np
import pytest

from oracle.coefficients import idx, multi_indices, n_moments, self_tensor
from oracle.rhs import lam_at, rhs_literal, rhs_regrouped, rk4


def _random_state(n, order, seed, spread=1.5, first_moments=True):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, 2)) * spread
    mom = rng.normal(size=(n, n_moments(order))) * 0.2
    mom[:, 0] = rng.choice([-1, 1], size=n) * (0.5 + rng.random(n))
    if not first_moments and order >= 1:
        mom[:, 1:3] = 0.0
    return x, mom


@pytest.mark.parametrize("order", [2, 4, 6, 10])
def test_axisymmetric_single_vortex_is_steady(order):
    mom = np.zeros((1, n_moments(order)))
    g = [1.0, 0.3, -0.2, 0.05, 0.01, -0.004]
    for a in range(order // 2 + 1):
        for b in range(order // 2 + 1 - a):
            mom[0, idx(2 * a, 2 * b)] = g[a + b] * math.comb(a + b, a)
    # size of the individual terms that must cancel: sum |T| |M_l| |M_m|
    scale = np.einsum("klm,l,m->k", np.abs(self_tensor(order, 0.9)), np.abs(mom[0]),
                      np.abs(mom[0])).max()
    dx, dM = rhs_regrouped(np.zeros((1, 2)), mom, 0.0, order, 0.9, 0.0)
    assert np.abs(dM).max() < 1e-15 * scale
    if order <= 4:
        dx, dM = rhs_literal(np.zeros((1, 2)), mom, 0.0, order, 0.9, 0.0)
        assert np.abs(dM).max() < 1e-15 * scale


def test_lamb_oseen_core_mismatch():
    lam0, mu0 = 2.0, 2.1
    d = mu0 ** 2 - lam0 ** 2
    errs = []
    for order in (0, 2, 4, 6, 8, 10, 12):
        mom = np.zeros((1, n_moments(order)))
        for a in range(order // 2 + 1):
            for b in range(order // 2 + 1 - a):
                mom[0, idx(2 * a, 2 * b)] = (d / 4) ** (a + b) / (math.factorial(a) * math.factorial(b))
        dx, dM = rhs_regrouped(np.zeros((1, 2)), mom, 8.0, order, lam0, 1e-3)
        assert np.abs(dM).max() < 1e-15
        # truncation error on a radial line: omega_M vs the true Gaussian
        r = np.linspace(0, 8, 161)
        lam = lam_at(8.0, lam0, 1e-3)
        mu = math.sqrt(lam ** 2 + d)
        true = np.exp(-r ** 2 / mu ** 2) / (math.pi * mu ** 2)
        approx = np.zeros_like(r)
        # Evaluate sum_n (d/4)^n/n! Lap^n phi_00 with Lap^n phi_00 =
        # (-4/lambda^2)^n n! L_n(r^2/lambda^2) phi_00 (Laguerre polynomials).
        from numpy.polynomial import laguerre
        phi00 = np.exp(-r ** 2 / lam ** 2) / (math.pi * lam ** 2)
        for nn in range(order // 2 + 1):
            coef = np.zeros(nn + 1)
            coef[nn] = 1.0
            lap_n = (-4.0 / lam ** 2) ** nn * math.factorial(nn) * laguerre.lagval(r ** 2 / lam ** 2, coef) * phi00
            approx += (d / 4) ** nn / math.factorial(nn) * lap_n
        errs.append(np.abs(approx - true).max() / true.max())
    errs = np.array(errs)
    assert np.all(np.diff(np.log(errs)) < -1.0)     # geometric decrease in M


@pytest.mark.parametrize("order", [2, 3, 4])
def test_conservation_laws(order):
    x, mom = _random_state(6, order, 7 + order, first_moments=True)
    dx, dM = rhs_regrouped(x, mom, 0.3, order, 0.7, 0.02)
    scale = np.abs(dM).max()
    assert np.abs(dM[:, 0]).max() <= 1e-14 * scale                 # P-3
    assert np.abs(dM[:, 1:3]).max() <= 1e-13 * scale               # P-4
    impulse = (mom[:, :1] * dx).sum(0)                              # P-5
    assert np.abs(impulse).max() <= 1e-13 * np.abs(mom[:, :1] * dx).max()


def test_core_spreading_pair_rotation():
    g1, g2 = 1.0, 0.6
    lam0, nu = 0.5, 0.01
    x0 = np.array([[-0.6, 0.0], [0.6, 0.0]])
    mom = np.array([[g1], [g2]])
    T, nsteps = 2.0, 200
    x, m, t = rk4(x0, mom, 0.0, T / nsteps, nsteps, 0, lam0, nu)
    d = 1.2
    tt = np.linspace(0, T, 20001)
    om = (g1 + g2) / (2 * math.pi * d * d) * (1 - np.exp(-d * d / (2 * (lam0 ** 2 + 4 * nu * tt))))
    theta = np.trapezoid(om, tt)
    sep = x[0] - x[1]
    assert np.hypot(*sep) == pytest.approx(d, rel=1e-9)
    ang = math.atan2(sep[1], sep[0]) - math.pi
    ang = (ang + math.pi) % (2 * math.pi) - math.pi
    assert ang == pytest.approx(theta, rel=1e-7)
    # the centre of vorticity does not move
    cv = (g1 * x[0] + g2 * x[1]) / (g1 + g2)
    cv0 = (g1 * x0[0] + g2 * x0[1]) / (g1 + g2)
    assert np.abs(cv - cv0).max() < 1e-12


def _rotate(x, mom, order):
    xr = np.stack([-x[:, 1], x[:, 0]], axis=1)
    mr = np.zeros_like(mom)
    for a, b in multi_indices(order):
        mr[:, idx(a, b)] = (-1) ** a * mom[:, idx(b, a)]
    return xr, mr


def _reflect(x, mom, order):
    xr = np.stack([x[:, 0], -x[:, 1]], axis=1)
    mr = np.zeros_like(mom)
    for a, b in multi_indices(order):
        mr[:, idx(a, b)] = -(-1) ** b * mom[:, idx(a, b)]
    return xr, mr


@pytest.mark.parametrize("order", [3, 4])
def test_rotation_and_reflection_covariance(order):
    x, mom = _random_state(5, order, 21)
    dx, dM = rhs_regrouped(x, mom, 0.1, order, 0.8, 0.01)
    for fn in (_rotate, _reflect):
        x2, m2 = fn(x, mom, order)
        dx2, dM2 = rhs_regrouped(x2, m2, 0.1, order, 0.8, 0.01)
        ex, eM = fn(dx, dM, order)
        assert np.abs(dM2 - eM).max() <= 1e-13 * np.abs(dM).max()
        assert np.abs(dx2 - ex).max() <= 1e-13 * np.abs(dx).max()


def test_rk4_fourth_order():
    x, mom = _random_state(3, 2, 31, spread=1.0, first_moments=False)
    ref = rk4(x, mom, 0.0, 0.4 / 64, 64, 2, 0.6, 0.05)
    errs = []
    for nsteps in (4, 8, 16):
        xs, ms, _ = rk4(x, mom, 0.0, 0.4 / nsteps, nsteps, 2, 0.6, 0.05)
        errs.append(max(np.abs(xs - ref[0]).max(), np.abs(ms - ref[1]).max()))
    r1 = errs[0] / errs[1]
    r2 = errs[1] / errs[2]
    assert 12 < r1 < 20 and 12 < r2 < 20
