"""Pins for the oracle's coefficient tables (closed forms of Appendix A.1).

* H_1, H_2 (the displays after eq:Fullint) against an independent derivation:
  V_00(b; sqrt2 lambda) = grad-perp psi with the stream function of a Gaussian
  vortex, whose Taylor series at 0 is psi = -(1/4pi) sum_{k>=1} (-x)^k / (k k!)
  with x = |b|^2/(2 lambda^2)  (psi = (ln x + E_1(x))/(4 pi) + const).  So
  H_1(a) = -D^{a+e2} psi(0), H_2(a) = D^{a+e1} psi(0), computed here in exact
  rational arithmetic for |a| <= 12 and compared with the stored golden table
  (written by tests/golden/make_golden.py from the oracle) and the oracle.
* c_k (eq:coefficient) against brute-force projection of Hermite functions:
  P_k[phi_m] = delta_km.
* The coefficient tensor c_k Gamma-tilde: the parity rule (nonzero only when
  k1+l1+m1 and k2+l2+m2 are both odd) and its lambda-homogeneity
  T(lambda) = T(1) lambda^{|k|-|l|-|m|-2} (direct build at lambda != 1).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle.coefficients import (H1, H2, _h_rational, c_k, gamma_tensor, idx,
                                 jet_table_at_zero, multi_indices, self_tensor)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "h_closed_forms.txt")


def _psi_derivative_at_zero(a1, a2):
    """D^(a1,a2) psi(0) / [(1/2pi) (2 lambda^2)^{-(a1+a2)/2}] as an exact rational.

    psi(b) = -(1/4pi) sum_k (-1)^k (b1^2+b2^2)^k / (k k! c^k), c = 2 lambda^2.
    The coefficient of b1^{a1} b2^{a2} is nonzero only for a1, a2 even; then
    k = (a1+a2)/2 and it equals -(1/4pi)(-1)^k C(k, a1/2)/(k k! c^k).
    D^a psi(0) = a1! a2! * that coefficient.
    """
    if a1 % 2 or a2 % 2 or a1 + a2 == 0:
        return Fraction(0)
    k = (a1 + a2) // 2
    # -(1/4pi) = (1/2pi) * (-1/2)
    return Fraction(-1, 2) * (-1) ** k * math.comb(k, a1 // 2) * math.factorial(a1) \
        * math.factorial(a2) / Fraction(k * math.factorial(k))


def test_h_closed_forms_equal_stream_function_series():
    for n in range(0, 13):
        for a2 in range(n + 1):
            a1 = n - a2
            # H_1(a) = -D^{a+e2} psi(0): both carry (1/2pi) (2 lambda^2)^{-(n+1)... }
            assert _h_rational(a1, a2, 1) == -_psi_derivative_at_zero(a1, a2 + 1)
            assert _h_rational(a1, a2, 2) == _psi_derivative_at_zero(a1 + 1, a2)


def test_h_golden_table():
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 2 * 91
    for comp, a1, a2, num, den in rows:
        assert Fraction(int(num), int(den)) == _h_rational(int(a1), int(a2), int(comp))
    # and the float evaluation at a non-unit lambda
    lam = 0.37
    for comp, a1, a2, num, den in rows:
        n = (int(a1) + int(a2) - 1) // 2
        ref = float(Fraction(int(num), int(den))) / (2 * math.pi) * (2 * lam * lam) ** (-(n + 1)) \
            if int(num) else 0.0
        got = (H1 if comp == "1" else H2)(int(a1), int(a2), lam)
        assert got == pytest.approx(ref, rel=1e-15, abs=0.0)


def test_ck_projects_hermite_functions():
    lam = 0.8
    npts = 240
    h = 16 * lam / npts
    g = (np.arange(npts) + 0.5) * h - 8 * lam
    Z1, Z2 = np.meshgrid(g, g, indexing="ij")
    phi00 = np.exp(-(Z1 ** 2 + Z2 ** 2) / lam ** 2) / (math.pi * lam ** 2)

    def hs(n, z):
        coef = np.zeros(n + 1)
        coef[n] = 1.0
        return np.polynomial.hermite.hermval(z / lam, coef) / lam ** n

    for k1, k2 in multi_indices(4):
        for m1, m2 in multi_indices(4):
            phim = (-1) ** (m1 + m2) * hs(m1, Z1) * hs(m2, Z2) * phi00
            val = c_k(k1, k2, lam) * (hs(k1, Z1) * hs(k2, Z2) * phim).sum() * h * h
            assert val == pytest.approx(1.0 if (k1, k2) == (m1, m2) else 0.0, abs=1e-11)


@pytest.mark.parametrize("order", [2, 4, 5])
def test_tensor_parity_and_homogeneity(order):
    T1 = self_tensor(order, 1.0)
    mi = multi_indices(order)
    for ki, (k1, k2) in enumerate(mi):
        for li, (l1, l2) in enumerate(mi):
            for mj, (m1, m2) in enumerate(mi):
                if T1[ki, li, mj] != 0.0:
                    assert (k1 + l1 + m1) % 2 == 1 and (k2 + l2 + m2) % 2 == 1
    assert np.count_nonzero(T1) > 0
    lam = 0.63
    J1, J2 = jet_table_at_zero(3 * order - 1, lam)
    direct = gamma_tensor(order, lam, J1, J2)
    scaled = self_tensor(order, lam)
    assert np.abs(direct - scaled).max() <= 1e-13 * np.abs(direct).max()


@pytest.mark.parametrize("order", [2, 4])
def test_finish_term_scaling(order):
    """The regrouped form's term list at lambda equals a direct build at lambda."""
    from oracle.coefficients import c_k, gamma_I_terms, gamma_II_terms
    from oracle.rhs import _finish_terms

    lam = 0.77
    ks, ls, cs, comps, offs = _finish_terms(order, lam)
    direct = []
    for ki, (k1, k2) in enumerate(multi_indices(order)):
        for li, (l1, l2) in enumerate(multi_indices(order)):
            for terms in (gamma_I_terms(k1, k2, l1, l2, lam), gamma_II_terms(k1, k2, l1, l2, lam)):
                for coef, _ in terms:
                    direct.append(c_k(k1, k2, lam) * coef)
    np.testing.assert_allclose(cs, np.array(direct), rtol=1e-14, atol=0)
