"""The paper's first convergence study (Section 4.1.1) on the GPU: a
Lamb-Oseen vortex of true core mu_0 = 2.1 expanded at lambda_0 = 2, Re = 1000,
single particle at orders 0 .. 24 (table finish up to 16, the separable self
term above), integrated with mmvm_integrate to t = 2, 4, 8, 16, 32 and
rebuilt with mmvm_vorticity.

The exact solution is the Gaussian of core mu(t)^2 = lambda(t)^2 + d,
d = mu_0^2 - lambda_0^2, whose expansion M_(2a,2b) = (d/4)^{a+b}/(a! b!) is
stationary under the MMVM.  Checked: the state stays put; the rebuilt field
equals the truncated series (written with Laguerre polynomials,
Lap^n phi_00 = (-4/lambda^2)^n n! L_n(r^2/lambda^2) phi_00) to rounding; and
the relative L-infinity error against the true Gaussian falls geometrically
in the order (the straight line of the paper's figure) until it reaches the
FP64 floor.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import laguerre

from oracle.rhs import lam_at

pytestmark = pytest.mark.gpu

LAM0, MU0, NU = 2.0, 2.1, 1e-3
ORDERS = (0, 2, 4, 6, 8, 12, 16, 20, 24)
TIMES = (2.0, 4.0, 8.0, 16.0, 32.0)


@pytest.fixture(scope="module")
def mm():
    import paper_1010_2475_gb300 as mm

    mm.load_library()
    return mm


def _moments(order):
    d = MU0 ** 2 - LAM0 ** 2
    K = (order + 1) * (order + 2) // 2
    m = np.zeros((1, K))
    for a in range(order // 2 + 1):
        for b in range(order // 2 + 1 - a):
            n = 2 * a + 2 * b
            m[0, n * (n + 1) // 2 + 2 * b] = (d / 4) ** (a + b) / (
                math.factorial(a) * math.factorial(b))
    return m


def _points():
    r = np.linspace(0.0, 14.0, 281)
    pts = [np.stack([r * math.cos(th), r * math.sin(th)], axis=1)
           for th in (0.0, math.pi / 7, math.pi / 4)]
    return np.concatenate(pts), np.concatenate([r, r, r])


def _truncated(order, lam, r):
    d = MU0 ** 2 - LAM0 ** 2
    phi00 = np.exp(-r ** 2 / lam ** 2) / (math.pi * lam ** 2)
    out = np.zeros_like(r)
    for n in range(order // 2 + 1):
        c = np.zeros(n + 1)
        c[n] = 1.0
        lap_n = (-4.0 / lam ** 2) ** n * math.factorial(n) * laguerre.lagval(r ** 2 / lam ** 2, c)
        out += (d / 4) ** n / math.factorial(n) * lap_n * phi00
    return out


def test_lamb_oseen_convergence_curve(mm):
    pts, r = _points()
    errs = {}
    for order in ORDERS:
        m0 = _moments(order)
        with mm.Context(order, LAM0, NU, mm.MMVM_FP64) as ctx:
            ctx.set_state(np.zeros((1, 2)), m0, 0.0)
            for T in TIMES:
                ctx.integrate(T, h0=0.1, rtol=1e-10, atol=1e-12)
                x, m, t = ctx.get_state()
                assert t == T and np.all(x == 0.0)
                assert np.abs(m - m0).max() <= 1e-13  # stationary
                w = ctx.vorticity(pts)
                lam = lam_at(T, LAM0, NU)
                mu = math.sqrt(lam ** 2 + MU0 ** 2 - LAM0 ** 2)
                true = np.exp(-r ** 2 / mu ** 2) / (math.pi * mu ** 2)
                series = _truncated(order, lam, r)
                assert np.abs(w - series).max() <= 1e-12 * true.max()
                errs[order, T] = np.abs(w - true).max() / true.max()
    for T in TIMES:
        e = np.array([errs[o, T] for o in ORDERS])
        above = e > 1e-12
        # geometric decrease while above the FP64 floor: every two orders cut
        # the error by more than 5x (about 10x for this core ratio), and
        # log10(e) is a straight line in the order (slope about -0.5)
        for a, b, oa, ob in zip(e, e[1:], ORDERS, ORDERS[1:]):
            if b > 1e-12:
                assert b < a * 0.2 ** ((ob - oa) / 2)
        o = np.array(ORDERS)[above]
        slope, icpt = np.polyfit(o, np.log10(e[above]), 1)
        resid = np.log10(e[above]) - (slope * o + icpt)
        assert slope < -0.4 and np.abs(resid).max() < 1.0
        assert e[-1] < 1e-12
