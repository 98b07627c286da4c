"""Exact rows of the single-particle moment equation (oracle, rational).

Test infrastructure only (see ``oracle/__init__.py``).

For one particle the right-hand side is the self term alone
(eq:moment_evolutionFinish): dM_k/dt = c_k sum_l M_l [Gamma^I + Gamma^II],
the (i, q) double sums of eq:FinalSingleI / eq:FinalSingleII with the
closed forms H_1, H_2 of Appendix A.1.  At lambda = 1 every factor is
rational except the 1/(2 pi) of H_1 and H_2, which multiplies every term:
c_k = (-1)^{|k|} 2^{-|k|} / (k1! k2!), the bracketed factorial ratios are
integers times powers of 2, and H = r / (2 pi) 2^{-(n+1)} with r the exact
rational of ``coefficients._h_rational``.  A state whose moments are binary
floats is rational too, so 2 pi dM_k/dt is an exact rational: this module
evaluates it with ``fractions.Fraction``, following the paper's sums in the
same order as ``rhs.self_rhs_rows`` (velocity jet first,
W_c[gamma] = sum_m M_m H_c(m + gamma), then the (i, q) terms).  No rounding
happens before the final division by 2 pi, so the rows are exact to the
precision of that one division; they pin the FP64 evaluations at high order,
where the condition number of a row (sum of the absolute terms over the
result) reaches 1e16 and FP64 cannot certify itself.

Cost: a few seconds per row at order 60 (hundreds of thousands of rational
terms); only sampled rows are evaluated.
"""
from __future__ import annotations

import math
from fractions import Fraction

from .coefficients import _h_rational, idx, multi_indices


def _h_exact(a1: int, a2: int, comp: int) -> Fraction:
    """2 pi H_comp(a1, a2) at lambda = 1 (exact)."""
    r = _h_rational(a1, a2, comp)
    if r == 0:
        return Fraction(0)
    n = (a1 + a2 - 1) // 2
    return r / (2 ** (n + 1))


def _c_exact(k1: int, k2: int) -> Fraction:
    """c_k at lambda = 1 (eq:coefficient): (-1)^{|k|} 2^{-|k|} / (k1! k2!)."""
    n = k1 + k2
    return Fraction((-1) ** n, 2 ** n * math.factorial(k1) * math.factorial(k2))


def _falling(k: int, j: int) -> int:
    """k! / (k - j)! (0 when j > k)."""
    if j > k:
        return 0
    out = 1
    for t in range(k - j + 1, k + 1):
        out *= t
    return out


def self_rows_exact(mom_row, order: int, krows):
    """2 pi dM_k/dt (exact Fractions) and 2 pi S_k (the sum of the absolute
    values of the same terms, exact) for the moment rows ``krows`` of a
    single particle at lambda = 1 (eq:FinalSingleI/II, eq:coefficient,
    Appendix A.1 closed forms)."""
    mi = multi_indices(order)
    M = [Fraction(float(v)) for v in mom_row]
    nz = [(c, m) for c, m in enumerate(mi) if M[c] != 0]
    # velocity jets W_c[gamma] = sum_m M_m 2 pi H_c(m + gamma), |gamma| <= 2M - 1
    W = ({}, {})
    Wabs = ({}, {})
    for g in multi_indices(max(2 * order - 1, 0)):
        for comp in (0, 1):
            s = Fraction(0)
            a = Fraction(0)
            for c, (m1, m2) in nz:
                h = _h_exact(m1 + g[0], m2 + g[1], comp + 1)
                if h:
                    t = M[c] * h
                    s += t
                    a += abs(t)
            W[comp][g] = s
            Wabs[comp][g] = a
    vals, sums = [], []
    for kc in krows:
        k1, k2 = mi[kc]
        ck = _c_exact(k1, k2)
        tot = Fraction(0)
        ab = Fraction(0)
        for lc, (l1, l2) in nz:
            ml = M[lc]
            sgn = (-1) ** (l1 + l2)
            # Gamma^I: H_1 at m + (k1 + l1 - 2i - 1, k2 + l2 - 2q)
            if k1 >= 1:
                for i in range(0, min(l1, k1 - 1) + 1):
                    a = math.comb(l1, i) * 2 ** (i + 1) * _falling(k1, i + 1)
                    for q in range(0, min(l2, k2) + 1):
                        b = math.comb(l2, q) * 2 ** q * _falling(k2, q)
                        f = ck * sgn * a * b * ml
                        g = (k1 + l1 - 2 * i - 1, k2 + l2 - 2 * q)
                        tot += f * W[0][g]
                        ab += abs(f) * Wabs[0][g]
            # Gamma^II: H_2 at m + (k1 + l1 - 2i, k2 + l2 - 2q - 1)
            if k2 >= 1:
                for i in range(0, min(l1, k1) + 1):
                    a = math.comb(l1, i) * 2 ** i * _falling(k1, i)
                    for q in range(0, min(l2, k2 - 1) + 1):
                        b = math.comb(l2, q) * 2 ** (q + 1) * _falling(k2, q + 1)
                        f = ck * sgn * a * b * ml
                        g = (k1 + l1 - 2 * i, k2 + l2 - 2 * q - 1)
                        tot += f * W[1][g]
                        ab += abs(f) * Wabs[1][g]
        vals.append(tot)
        sums.append(ab)
    return vals, sums


def to_float(fr: Fraction, two_pi_digits: int = 40) -> float:
    """A Fraction 2 pi v divided by 2 pi, rounded once to the nearest float."""
    from decimal import Decimal, getcontext

    getcontext().prec = two_pi_digits + 10
    # pi to 50 digits
    pi = Decimal("3.14159265358979323846264338327950288419716939937510")
    return float(Decimal(fr.numerator) / Decimal(fr.denominator) / (2 * pi))


__all__ = ["self_rows_exact", "to_float", "idx"]
