"""Combinatorial coefficients of the MMVM moment ODE (oracle, FP64).

Test infrastructure only (see ``oracle/__init__.py``).

Notation follows the paper: k = (k1, k2) is the projected moment, l the
moment whose derivatives fall on the vorticity (the binomial index of the
integration by parts), m the moment carried by the velocity field.
lambda is the Gaussian core size, lambda^2 = lambda_0^2 + 4 nu t (eq:phi00).
"""
from __future__ import annotations

import math
from fractions import Fraction
from functools import lru_cache

import numpy as np

TWO_PI = 2.0 * math.pi


def n_moments(order: int) -> int:
    """K = (M+1)(M+2)/2 moments with k1 + k2 <= M (Section 2.1.2 truncation)."""
    return (order + 1) * (order + 2) // 2


def idx(k1: int, k2: int) -> int:
    """Column of moment (k1, k2): grouped by total order n, then by k2."""
    n = k1 + k2
    return n * (n + 1) // 2 + k2


@lru_cache(maxsize=None)
def multi_indices(order: int) -> tuple:
    """All (k1, k2) with k1 + k2 <= order, in column order."""
    return tuple((n - k2, k2) for n in range(order + 1) for k2 in range(n + 1))


def c_k(k1: int, k2: int, lam: float) -> float:
    """Projection prefactor of eq:coefficient:
    (-1)^{|k|} lambda^{2|k|} / (2^{|k|} k1! k2!)."""
    n = k1 + k2
    return (-1) ** n * (lam * lam / 2.0) ** n / (math.factorial(k1) * math.factorial(k2))


@lru_cache(maxsize=None)
def _h_rational(a1: int, a2: int, comp: int) -> Fraction:
    """Exact rational part of H_1 (comp=1) or H_2 (comp=2).

    Appendix A.1 (the two displays defining calligraphic H_1 and H_2):
      H_1(a) = -(1/2pi) (1/(2 lambda^2))^{n+1} (-1)^n / (n+1)! C(n, a1/2) a1! a2!
               for a1 even, a2 odd, n = (a1 + a2 - 1)/2, else 0;
      H_2(a) = +(1/2pi) (1/(2 lambda^2))^{n+1} (-1)^n / (n+1)! C(n, (a1-1)/2) a1! a2!
               for a1 odd, a2 even, else 0.
    Returned without the (1/2pi) and (2 lambda^2)^{-(n+1)} factors.
    """
    if comp == 1:
        if a1 % 2 != 0 or a2 % 2 != 1:
            return Fraction(0)
        n = (a1 + a2 - 1) // 2
        sign = -1
        kk = a1 // 2
    else:
        if a1 % 2 != 1 or a2 % 2 != 0:
            return Fraction(0)
        n = (a1 + a2 - 1) // 2
        sign = 1
        kk = (a1 - 1) // 2
    num = sign * (-1) ** n * math.comb(n, kk) * math.factorial(a1) * math.factorial(a2)
    return Fraction(num, math.factorial(n + 1))


def H1(a1: int, a2: int, lam: float) -> float:
    """H_1(a1, a2; lambda) = D^a V_00^1(b; sqrt(2) lambda) at b = 0."""
    r = _h_rational(a1, a2, 1)
    if r == 0:
        return 0.0
    n = (a1 + a2 - 1) // 2
    return float(r) / TWO_PI * (2.0 * lam * lam) ** (-(n + 1))


def H2(a1: int, a2: int, lam: float) -> float:
    """H_2(a1, a2; lambda) = D^a V_00^2(b; sqrt(2) lambda) at b = 0."""
    r = _h_rational(a1, a2, 2)
    if r == 0:
        return 0.0
    n = (a1 + a2 - 1) // 2
    return float(r) / TWO_PI * (2.0 * lam * lam) ** (-(n + 1))


def jet_table_at_zero(P: int, lam: float):
    """H_1, H_2 for all |alpha| <= P as (J1, J2) arrays in column order."""
    mi = multi_indices(P)
    J1 = np.array([H1(a1, a2, lam) for a1, a2 in mi])
    J2 = np.array([H2(a1, a2, lam) for a1, a2 in mi])
    return J1, J2


def _ratio(k: int, j: int) -> float:
    """k!/(k-j)! (falling factorial), 0 when j > k."""
    if j > k:
        return 0.0
    out = 1.0
    for t in range(k - j + 1, k + 1):
        out *= t
    return out


def gamma_I_terms(k1, k2, l1, l2, lam):
    """The (i, q) terms of Gamma^I (eq:FinalSingleI) as a list of
    (coefficient, offset) where the H_1 argument is m + offset.

    Gamma^I = sum_{i=0}^{min(l1,k1-1)} sum_{q=0}^{min(l2,k2)} C(l1,i) C(l2,q)
              (-1)^{l1+l2} [2^{i+1} k1! / (lambda^{2(i+1)} (k1-i-1)!)]
              [2^q k2! / (lambda^{2q} (k2-q)!)]
              H_1(m1 + k1 - i - 1 + l1 - i, m2 + k2 - q + l2 - q).
    """
    out = []
    if k1 < 1:
        return out
    s = (-1) ** (l1 + l2)
    for i in range(0, min(l1, k1 - 1) + 1):
        a = 2.0 ** (i + 1) * _ratio(k1, i + 1) / lam ** (2 * (i + 1))
        for q in range(0, min(l2, k2) + 1):
            b = 2.0 ** q * _ratio(k2, q) / lam ** (2 * q)
            coef = math.comb(l1, i) * math.comb(l2, q) * s * a * b
            out.append((coef, (k1 + l1 - 2 * i - 1, k2 + l2 - 2 * q)))
    return out


def gamma_II_terms(k1, k2, l1, l2, lam):
    """The (i, q) terms of Gamma^II (eq:FinalSingleII), H_2 argument m + offset.

    Gamma^II = sum_{i=0}^{min(l1,k1)} sum_{q=0}^{min(l2,k2-1)} C(l1,i) C(l2,q)
               (-1)^{l1+l2} [2^i k1! / (lambda^{2i} (k1-i)!)]
               [2^{q+1} k2! / (lambda^{2(q+1)} (k2-q-1)!)]
               H_2(m1 + k1 - i + l1 - i, m2 + k2 - q - 1 + l2 - q).
    """
    out = []
    if k2 < 1:
        return out
    s = (-1) ** (l1 + l2)
    for i in range(0, min(l1, k1) + 1):
        a = 2.0 ** i * _ratio(k1, i) / lam ** (2 * i)
        for q in range(0, min(l2, k2 - 1) + 1):
            b = 2.0 ** (q + 1) * _ratio(k2, q + 1) / lam ** (2 * (q + 1))
            coef = math.comb(l1, i) * math.comb(l2, q) * s * a * b
            out.append((coef, (k1 + l1 - 2 * i, k2 + l2 - 2 * q - 1)))
    return out


def gamma_tensor(order: int, lam: float, J1: np.ndarray, J2: np.ndarray) -> np.ndarray:
    """Literal coefficient tensor T[k, l, m] = c_k (Gamma^I + Gamma^II)[k, l, m].

    J1, J2 hold the first / second velocity-component kernel for every
    |alpha| <= 3*order - 1 in column order: the closed forms H_1, H_2 for the
    single-vortex coefficient Gamma-tilde (eq:moment_evolutionFinish), or the
    pair kernel H^B_1, H^B_2 at a separation s for Gamma_B (eq:FinalCrossI/II).
    dM_k/dt gets sum_{l,m} T[k,l,m] M_l M_m (l: vorticity index, m: velocity).
    """
    mi = multi_indices(order)
    K = len(mi)
    T = np.zeros((K, K, K))
    m1 = np.array([m[0] for m in mi])
    m2 = np.array([m[1] for m in mi])
    for ki, (k1, k2) in enumerate(mi):
        ck = c_k(k1, k2, lam)
        for li, (l1, l2) in enumerate(mi):
            acc = np.zeros(K)
            for coef, (o1, o2) in gamma_I_terms(k1, k2, l1, l2, lam):
                a1 = m1 + o1
                a2 = m2 + o2
                acc += coef * J1[(a1 + a2) * (a1 + a2 + 1) // 2 + a2]
            for coef, (o1, o2) in gamma_II_terms(k1, k2, l1, l2, lam):
                a1 = m1 + o1
                a2 = m2 + o2
                acc += coef * J2[(a1 + a2) * (a1 + a2 + 1) // 2 + a2]
            T[ki, li, :] = ck * acc
    return T


@lru_cache(maxsize=8)
def self_tensor_unit(order: int) -> np.ndarray:
    """c_k Gamma-tilde at lambda = 1 (cached; see ``self_tensor``)."""
    J1, J2 = jet_table_at_zero(3 * order - 1 if order > 0 else 0, 1.0)
    T = gamma_tensor(order, 1.0, J1, J2)
    T.setflags(write=False)
    return T


def self_tensor(order: int, lam: float) -> np.ndarray:
    """c_k Gamma-tilde[k,l,m] at core size lambda.

    Built once at lambda = 1 and rescaled by lambda^{|k|-|l|-|m|-2}: every
    factor of eq:FinalSingleI/II and eq:coefficient is a power of lambda
    (c_k ~ lambda^{2|k|}, the bracketed ratios ~ lambda^{-2(i+q+1)}, H ~
    lambda^{-(|alpha|+1)} with |alpha| = |k|+|l|+|m|-2(i+q)-1).  The identity
    is pinned against a direct build in the tests.
    """
    T1 = self_tensor_unit(order)
    if lam == 1.0:
        return np.array(T1)
    n = np.array([a + b for a, b in multi_indices(order)])
    p = n[:, None, None] - n[None, :, None] - n[None, None, :] - 2
    return T1 * lam ** p
