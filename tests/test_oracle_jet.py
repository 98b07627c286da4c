"""Pins for the oracle's pair kernel H^B(alpha; s) (Appendix A.2).

* s -> 0: equals the closed forms H_1, H_2 (a different formula entirely).
* 60-digit reference: D^a of F(|zeta|^2) by the Faa di Bruno expansion with
  F^{(n)}(x) = (-1)^n gamma(n+1, x)/x^{n+1} in mpmath, on both sides of the
  oracle's near/far switch and for orders up to 26.
* Field identities of the velocity of a Gaussian vortex of core sqrt2 lambda:
  divergence free (J1[a+e1] + J2[a+e2] = 0) and curl equal to its vorticity
  (J2[a+e1] - J1[a+e2] = D^a exp(-|b|^2/c)/(pi c), a product of Hermite
  functions), for every entry.
* Antisymmetry J(-s) = (-1)^{|a|+1} J(s) (V_00 is odd).
* Far field: the point-vortex jet i^{a2} (-i/2pi)(-1)^n n!/z^{n+1}.
"""
import math

import numpy as np
import pytest

from oracle.coefficients import idx, jet_table_at_zero, multi_indices
from oracle.pair_jet import pair_jet


def _order_scaled_err(J1, J2, R1, R2, P):
    worst = 0.0
    for n in range(P + 1):
        cols = [idx(n - a2, a2) for a2 in range(n + 1)]
        sc = max(np.abs(R1[..., cols]).max(), np.abs(R2[..., cols]).max(), 1e-300)
        e = max(np.abs(J1[..., cols] - R1[..., cols]).max(),
                np.abs(J2[..., cols] - R2[..., cols]).max()) / sc
        worst = max(worst, e)
    return worst


def test_zero_separation_equals_closed_forms():
    for P, lam in ((11, 1.0), (17, 0.45), (23, 2.0)):
        H1t, H2t = jet_table_at_zero(P, lam)
        J1, J2 = pair_jet(np.zeros((1, 2)), P, lam)
        assert _order_scaled_err(J1[0], J2[0], H1t, H2t, P) < 1e-13


def test_against_60_digit_reference():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60

    def I_n(n, x):
        return mp.mpf(1) / (n + 1) if x == 0 else mp.gammainc(n + 1, 0, x) / x ** (n + 1)

    def dF(a1, a2, z1, z2):
        x = z1 * z1 + z2 * z2
        tot = mp.mpf(0)
        for k in range(a1 // 2 + 1):
            for l in range(a2 // 2 + 1):
                coef = (mp.factorial(a1) * mp.factorial(a2)
                        / (mp.factorial(k) * mp.factorial(a1 - 2 * k)
                           * mp.factorial(l) * mp.factorial(a2 - 2 * l)))
                nn = a1 + a2 - k - l
                tot += coef * (2 * z1) ** (a1 - 2 * k) * (2 * z2) ** (a2 - 2 * l) \
                    * (-1) ** nn * I_n(nn, x)
        return tot

    def ref(s1, s2, P, lam):
        c = 2 * mp.mpf(lam) ** 2
        rc = mp.sqrt(c)
        z1, z2 = mp.mpf(s1) / rc, mp.mpf(s2) / rc
        out1, out2 = [], []
        for a1, a2 in multi_indices(P):
            n = a1 + a2
            g = dF(a1, a2, z1, z2) * c ** (-1 - mp.mpf(n) / 2)
            g2 = dF(a1, a2 - 1, z1, z2) * c ** (-1 - mp.mpf(n - 1) / 2) if a2 else 0
            g1 = dF(a1 - 1, a2, z1, z2) * c ** (-1 - mp.mpf(n - 1) / 2) if a1 else 0
            out1.append(-(mp.mpf(s2) * g + a2 * g2) / (2 * mp.pi))
            out2.append((mp.mpf(s1) * g + a1 * g1) / (2 * mp.pi))
        return np.array([float(v) for v in out1]), np.array([float(v) for v in out2])

    lam = 0.7
    c = 2 * lam * lam
    for P in (8, 17, 23):
        xs = max(2.5, 0.3 * P)
        for x in (0.01, 0.5, 0.9 * xs, 1.1 * xs, 30.0, 250.0, 2000.0):
            th = 0.37 + x
            r = math.sqrt(x * c)
            s = (r * math.cos(th), r * math.sin(th))
            R1, R2 = ref(s[0], s[1], P, lam)
            J1, J2 = pair_jet(np.array([s]), P, lam)
            assert _order_scaled_err(J1[0], J2[0], R1, R2, P) < 2e-13, (P, x)


@pytest.mark.parametrize("P", [7, 17])
def test_divergence_and_curl_identities(P):
    lam = 0.55
    c = 2 * lam * lam
    rng = np.random.default_rng(3)
    s = rng.normal(size=(40, 2)) * np.exp(rng.uniform(-3, 2.5, size=(40, 1)))
    J1, J2 = pair_jet(s, P, lam)
    zeta = s / math.sqrt(c)
    ex = np.exp(-(zeta ** 2).sum(1))

    def herm(k, y):
        coef = np.zeros(k + 1)
        coef[k] = 1.0
        return np.polynomial.hermite.hermval(y, coef)

    for a1, a2 in multi_indices(P - 1):
        n = a1 + a2
        scale = max(np.abs(J1[:, [idx(n + 1 - b, b) for b in range(n + 2)]]).max(), 1e-300)
        div = J1[:, idx(a1 + 1, a2)] + J2[:, idx(a1, a2 + 1)]
        assert np.abs(div).max() <= 1e-12 * scale
        curl = J2[:, idx(a1 + 1, a2)] - J1[:, idx(a1, a2 + 1)]
        vort = (c ** (-n / 2) * (-1) ** n * herm(a1, zeta[:, 0]) * herm(a2, zeta[:, 1])
                * ex / (math.pi * c))
        assert np.abs(curl - vort).max() <= 1e-12 * scale


def test_odd_symmetry_and_point_vortex_far_field():
    lam = 0.9
    P = 14
    rng = np.random.default_rng(4)
    s = rng.normal(size=(25, 2)) * 3
    J1, J2 = pair_jet(s, P, lam)
    K1, K2 = pair_jet(-s, P, lam)
    sign = np.array([(-1.0) ** (a + b + 1) for a, b in multi_indices(P)])
    assert np.abs(K1 - sign * J1).max() <= 1e-13 * np.abs(J1).max()
    assert np.abs(K2 - sign * J2).max() <= 1e-13 * np.abs(J2).max()
    far = rng.normal(size=(10, 2)) * 60 + 40
    F1, F2 = pair_jet(far, P, lam)
    z = far[:, 0] + 1j * far[:, 1]
    for a1, a2 in multi_indices(P):
        n = a1 + a2
        v = (1j) ** a2 * (-1j / (2 * math.pi)) * (-1) ** n * math.factorial(n) / z ** (n + 1)
        np.testing.assert_allclose(F1[:, idx(a1, a2)], v.real, rtol=1e-12, atol=1e-14 * np.abs(v).max())
        np.testing.assert_allclose(F2[:, idx(a1, a2)], -v.imag, rtol=1e-12, atol=1e-14 * np.abs(v).max())


def test_far_branch_equals_explicit_leibniz_loop():
    """The far branch of the oracle's jet (Toeplitz products of
    Taylor-normalised arrays) against the two-variable Leibniz rule written
    out term by term: D^a (V_pv - V_pv E) = D^a V_pv - sum_{b <= a}
    C(a1, b1) C(a2, b2) D^b V_pv D^{a-b} E, with D^b of the holomorphic
    V_pv,1 - i V_pv,2 = (-i/2pi)/z equal to i^{b2} (-i/2pi)(-1)^n n!/z^{n+1}
    (n = |b|) and D^c E a product of Hermite functions."""
    import math

    from oracle.coefficients import multi_indices
    from oracle.pair_jet import _far

    P, lam = 8, 0.7
    c = 2.0 * lam * lam
    s = np.array([[2.1, 0.4], [-1.3, 2.2], [0.2, -3.5], [4.0, 4.0]])

    def herm(k, y):
        h = [1.0, 2.0 * y]
        for j in range(1, k):
            h.append(2.0 * y * h[j] - 2.0 * j * h[j - 1])
        return h[k]

    def dE(c1, c2, b1, b2):  # D_1^c1 D_2^c2 exp(-(b1^2 + b2^2)/c)
        out = 1.0
        for k, b in ((c1, b1), (c2, b2)):
            t = b / math.sqrt(c)
            out *= c ** (-k / 2.0) * (-1.0) ** k * herm(k, t) * math.exp(-t * t)
        return out

    def dpv(b1, b2, z):  # (D^b V_pv,1, D^b V_pv,2)
        n = b1 + b2
        f = (1j) ** b2 * (-1j / (2.0 * math.pi)) * (-1.0) ** n * math.factorial(n) / z ** (n + 1)
        return f.real, -f.imag

    J1, J2 = _far(s, P, c)
    mi = multi_indices(P)
    for p, (s1, s2) in enumerate(s):
        z = s1 + 1j * s2
        for col, (a1, a2) in enumerate(mi):
            v1, v2 = dpv(a1, a2, z)
            for b1 in range(a1 + 1):
                for b2 in range(a2 + 1):
                    w = math.comb(a1, b1) * math.comb(a2, b2) * dE(a1 - b1, a2 - b2, s1, s2)
                    p1, p2 = dpv(b1, b2, z)
                    v1 -= w * p1
                    v2 -= w * p2
            n = a1 + a2
            scale = max(abs(J1[p, k]) + abs(J2[p, k]) for k, (q1, q2) in enumerate(mi)
                        if q1 + q2 == n)
            assert abs(J1[p, col] - v1) <= 1e-12 * scale
            assert abs(J2[p, col] - v2) <= 1e-12 * scale
