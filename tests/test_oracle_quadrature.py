"""Pin the oracle's right-hand side to brute-force quadrature of its definition.

The moment ODE of Section 2.2 (eq:mom_multi, eq:xjdot) is, for each particle
j and each |k| <= M,

  dM^j_k/dt = P_k[ -(sum_{j'} u^{j'}(z + s_jj')) . grad omega^j(z) ]
              + P_k[ xdot^j . grad omega^j(z) ],
  xdot^j   = (1/M^j_00) sum_{j' != j} int u^{j'}(z + s_jj') omega^j(z) dz,

with the projection P_k[f] = c_k int H_k(z; lambda) f(z) dz (eq:coefficient),
omega^j = sum_l M^j_l D^l phi_00 (eq:moment_expansion_def_tw0) and
u^{j'} = sum_m M^{j'}_m D^m V_00 (eq:velocity_field_expansion, eq:Vzerodef).
Here every integral is summed on a fine grid (trapezoid rule, spectrally
accurate for these Gaussian-weighted integrands) and the derivatives of V_00
come from sympy, so nothing of the oracle's combinatorics is reused.  The
orders tested are <= 3.

The same quadrature also shows that the two printed alternatives the oracle
does NOT take would be wrong: the separation s = x^{j'} - x^j, and the cross
term with M^{j'}_l M^j_m (the binomial index on the source particle).
"""
import math

import numpy as np
import pytest

sympy = pytest.importorskip("sympy")
mpmath = pytest.importorskip("mpmath")

from oracle.coefficients import c_k, gamma_tensor, idx, multi_indices, n_moments
from oracle.pair_jet import pair_jet
from oracle.rhs import lam_at, rhs_literal, rhs_regrouped


def _v00_derivative_functions(order, lam):
    """numpy and mpmath callables for D^m V_00(y; lambda), |m| <= order."""
    y1, y2 = sympy.symbols("y1 y2", real=True)
    r2 = y1 ** 2 + y2 ** 2
    g = (1 - sympy.exp(-r2 / sympy.Float(lam) ** 2)) / r2 / (2 * sympy.pi)
    V = (-y2 * g, y1 * g)
    fns = {}
    for m1, m2 in multi_indices(order):
        comps = []
        for c in range(2):
            e = V[c]
            if m1:
                e = sympy.diff(e, y1, m1)
            if m2:
                e = sympy.diff(e, y2, m2)
            comps.append((sympy.lambdify((y1, y2), e, "numpy"),
                          sympy.lambdify((y1, y2), e, "mpmath")))
        fns[(m1, m2)] = comps
    return fns


def _eval_V(fns, m, c, y1, y2, lam):
    """Evaluate D^m V_00,c on arrays, in 40-digit arithmetic near the origin."""
    f_np, f_mp = fns[m][c]
    out = np.asarray(f_np(y1, y2), dtype=np.float64) * np.ones_like(y1)
    near = (y1 * y1 + y2 * y2) < (0.3 * lam) ** 2
    if np.any(near):
        with mpmath.workdps(40):
            out[near] = [float(f_mp(mpmath.mpf(a), mpmath.mpf(b)))
                         for a, b in zip(y1[near], y2[near])]
    return out


def _hermite_scaled(n, z, lam):
    """H_n(z; lambda) = lambda^{-n} Hermite_n(z / lambda) in one variable."""
    coef = np.zeros(n + 1)
    coef[n] = 1.0
    return np.polynomial.hermite.hermval(z / lam, coef) / lam ** n


def _quadrature_rhs(x, mom, order, lam, s_sign=+1, npts=300, half_width=8.0):
    n = x.shape[0]
    fns = _v00_derivative_functions(order, lam)
    h = 2 * half_width * lam / npts
    g = (np.arange(npts) + 0.5) * h - half_width * lam      # no node at z = 0
    Z1, Z2 = np.meshgrid(g, g, indexing="ij")
    w = h * h
    phi00 = np.exp(-(Z1 ** 2 + Z2 ** 2) / lam ** 2) / (math.pi * lam ** 2)
    Hx = {k: _hermite_scaled(k, Z1, lam) for k in range(order + 3)}
    Hy = {k: _hermite_scaled(k, Z2, lam) for k in range(order + 3)}

    def phi(n1, n2):
        return (-1) ** (n1 + n2) * Hx[n1] * Hy[n2] * phi00

    dxdt = np.zeros((n, 2))
    dM = np.zeros((n, n_moments(order)))
    for j in range(n):
        om = sum(mom[j, idx(l1, l2)] * phi(l1, l2) for l1, l2 in multi_indices(order))
        gx = sum(mom[j, idx(l1, l2)] * phi(l1 + 1, l2) for l1, l2 in multi_indices(order))
        gy = sum(mom[j, idx(l1, l2)] * phi(l1, l2 + 1) for l1, l2 in multi_indices(order))
        u_all = [np.zeros_like(Z1), np.zeros_like(Z1)]
        u_other = [np.zeros_like(Z1), np.zeros_like(Z1)]
        for jp in range(n):
            s = s_sign * (x[j] - x[jp])
            Y1 = Z1 + s[0]
            Y2 = Z2 + s[1]
            for m1, m2 in multi_indices(order):
                for c in range(2):
                    v = mom[jp, idx(m1, m2)] * _eval_V(fns, (m1, m2), c, Y1, Y2, lam)
                    u_all[c] += v
                    if jp != j:
                        u_other[c] += v
        xd = np.array([(u_other[0] * om).sum() * w, (u_other[1] * om).sum() * w]) / mom[j, 0]
        dxdt[j] = xd
        adv = -(u_all[0] * gx + u_all[1] * gy) + xd[0] * gx + xd[1] * gy
        for k1, k2 in multi_indices(order):
            Hk = Hx[k1] * Hy[k2]
            dM[j, idx(k1, k2)] = c_k(k1, k2, lam) * (Hk * adv).sum() * w
    return dxdt, dM


def _state(order, seed):
    rng = np.random.default_rng(seed)
    x = np.array([[0.0, 0.0], [1.1, 0.4], [-0.3, 1.3]])
    K = n_moments(order)
    mom = rng.normal(size=(3, K)) * 0.15
    mom[:, 0] = [1.0, 0.7, -0.5]
    return x, mom


@pytest.mark.parametrize("order", [1, 2, 3])
def test_rhs_matches_biot_savart_quadrature(order):
    x, mom = _state(order, 11 + order)
    lam0, nu, t = 0.6, 0.01, 0.5
    lam = lam_at(t, lam0, nu)
    qx, qM = _quadrature_rhs(x, mom, order, lam)
    ox, oM = rhs_regrouped(x, mom, t, order, lam0, nu)
    lx, lM = rhs_literal(x, mom, t, order, lam0, nu)
    # order 1 has dM/dt = 0 identically (first moments are conserved), so the
    # moment scale is floored by the centroid-velocity scale.
    scale = max(np.abs(qM).max(), np.abs(qx).max() * np.abs(mom).max())
    assert np.abs(oM - qM).max() <= 1e-9 * scale
    assert np.abs(lM - qM).max() <= 1e-9 * scale
    assert np.abs(ox - qx).max() <= 1e-9 * np.abs(qx).max()
    assert np.abs(lx - qx).max() <= 1e-9 * np.abs(qx).max()


def test_printed_alternatives_fail_the_quadrature():
    """The readings the oracle takes are the only ones the quadrature accepts."""
    order = 2
    x, mom = _state(order, 5)
    lam0, nu, t = 0.6, 0.0, 0.0
    lam = lam0
    qx, qM = _quadrature_rhs(x, mom, order, lam)
    # (a) s = x^{j'} - x^j: the quadrature under that sign disagrees with the
    # oracle, and the oracle agrees with the quadrature under its own sign.
    qx_flip, qM_flip = _quadrature_rhs(x, mom, order, lam, s_sign=-1)
    ox, oM = rhs_regrouped(x, mom, t, order, lam0, nu)
    assert np.abs(oM - qM).max() <= 1e-9 * np.abs(qM).max()
    assert np.abs(oM - qM_flip).max() > 1e-2 * np.abs(qM).max()
    # (b) cross term with the labels as printed (M^{j'}_l M^j_m): rebuild B so.
    P = 3 * order - 1
    dM_alt = oM.copy()
    for j in range(3):
        for jp in range(3):
            if jp == j:
                continue
            J1, J2 = pair_jet((x[j] - x[jp])[None, :], P, lam)
            T_B = gamma_tensor(order, lam, J1[0], J2[0])
            dM_alt[j] -= np.einsum("klm,l,m->k", T_B, mom[j], mom[jp])
            dM_alt[j] += np.einsum("klm,l,m->k", T_B, mom[jp], mom[j])
    assert np.abs(dM_alt - qM).max() > 1e-2 * np.abs(qM).max()
