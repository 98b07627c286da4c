"""Cross-term kernel H^B(alpha; s) of the MMVM (oracle, FP64).

Test infrastructure only (see ``oracle/__init__.py``).

Appendix A.2 defines, for a separation s between two particles,
    H^B(alpha) = D_b^alpha (1/2pi) (-b2, b1)/|b|^2 (1 - exp(-|b|^2 / (2 lambda^2)))
evaluated at b = s: the alpha-th derivative of the velocity of a Gaussian
vortex of core sqrt(2) lambda (eq:Fullint with b = s instead of 0).  The paper
stops there and gives no closed form for s != 0.  Write c = 2 lambda^2 and
x = |s|^2 / c.  The oracle evaluates the defining derivative by plain calculus
in one of two exact ways, switching at x_s = max(2.5, 0.3 P) for a jet of
order P (both agree with a 60-digit evaluation to ~1e-13 of the largest
entry of each order, |alpha| <= 26, on either side of the switch; see
``tests/test_oracle_jet.py``):

Near (x < x_s): the core factor G(b) = (1 - e^{-|b|^2/c}) / |b|^2 equals
(1/c) int_0^1 exp(-t |b|^2 / c) dt, so with zeta = b / sqrt(c)
    D_b^a G = c^{-1-|a|/2} int_0^1 (-1)^{|a|} Q_{a1}(t; zeta1) Q_{a2}(t; zeta2)
                                    exp(-t |zeta|^2) dt,
Q_k(t; y) = t^{k/2} Hermite_k(sqrt(t) y) (Q_0 = 1, Q_1 = 2ty,
Q_{k+1} = 2ty Q_k - 2kt Q_{k-1}); the t-integral is summed by 72-point
Gauss-Legendre.  Leibniz on V_1 = -(1/2pi) b2 G, V_2 = (1/2pi) b1 G gives
    D^a V_1 = -(1/2pi)[b2 D^a G + a2 D^{a-e2} G],
    D^a V_2 = +(1/2pi)[b1 D^a G + a1 D^{a-e1} G].

Far (x >= x_s): V_00 = V_pv - V_pv E with the point-vortex field
V_pv = (1/2pi)(-b2, b1)/|b|^2 and E = exp(-|b|^2/c).  V_pv,1 - i V_pv,2 =
(-i/2pi)/z (z = b1 + i b2) is holomorphic, so D^a of it is
i^{a2} (-i/2pi) (-1)^n n! / z^{n+1} with n = |a|; D^a E is the product of two
Hermite functions; D^a (V_pv E) follows from the two-variable Leibniz rule.
Beyond x = 400 the Leibniz term is below 1e-60 of the point-vortex term and
is not formed.
"""
from __future__ import annotations

import math

import numpy as np

from .coefficients import multi_indices

X_NO_TAIL = 400.0
_LEG = np.polynomial.legendre.leggauss(72)
_CHUNK = 2048


def _q_table(t: np.ndarray, y: np.ndarray, kmax: int) -> np.ndarray:
    """Q_k(t; y) for k = 0..kmax; t, y broadcastable; result (..., kmax+1)."""
    t, y = np.broadcast_arrays(t, y)
    out = np.empty(t.shape + (kmax + 1,))
    out[..., 0] = 1.0
    if kmax >= 1:
        out[..., 1] = 2.0 * t * y
    for k in range(1, kmax):
        out[..., k + 1] = 2.0 * t * y * out[..., k] - 2.0 * k * t * out[..., k - 1]
    return out


def _near(s: np.ndarray, P: int, c: float):
    """Near regime: quadrature of the t-integral (c = 2 lambda^2)."""
    rc = math.sqrt(c)
    z1 = s[:, 0] / rc
    z2 = s[:, 1] / rc
    x = z1 * z1 + z2 * z2
    nodes, weights = _LEG
    t = 0.5 * (nodes + 1.0)[None, :]
    w = (0.5 * weights)[None, :] * np.exp(-x[:, None] * t)
    amax = P + 1
    q1 = _q_table(t, z1[:, None], amax)
    q2 = _q_table(t, z2[:, None], amax)
    dF = np.einsum("pn,pna,pnb->pab", w, q1, q2, optimize=True)
    ar = np.arange(amax + 1)
    dF *= ((-1.0) ** (ar[:, None] + ar[None, :]))[None]
    # D_b^a G = c^{-1 - |a|/2} D_zeta^a F
    dG = dF * (c ** (-1.0 - (ar[:, None] + ar[None, :]) / 2.0))[None]
    mi = multi_indices(P)
    J1 = np.empty((s.shape[0], len(mi)))
    J2 = np.empty((s.shape[0], len(mi)))
    b1 = s[:, 0]
    b2 = s[:, 1]
    for col, (a1, a2) in enumerate(mi):
        g = dG[:, a1, a2]
        g_m2 = dG[:, a1, a2 - 1] if a2 >= 1 else 0.0
        g_m1 = dG[:, a1 - 1, a2] if a1 >= 1 else 0.0
        J1[:, col] = -(b2 * g + a2 * g_m2) / (2.0 * math.pi)
        J2[:, col] = (b1 * g + a1 * g_m1) / (2.0 * math.pi)
    return J1, J2


def _hermite(kmax: int, y: np.ndarray) -> np.ndarray:
    """Physicists' Hermite polynomials H_0..H_kmax at y; shape (n, kmax+1)."""
    out = np.empty(y.shape + (kmax + 1,))
    out[..., 0] = 1.0
    if kmax >= 1:
        out[..., 1] = 2.0 * y
    for k in range(1, kmax):
        out[..., k + 1] = 2.0 * y * out[..., k] - 2.0 * k * out[..., k - 1]
    return out


def _far(s: np.ndarray, P: int, c: float):
    """Far regime: point-vortex jet minus the Leibniz product with exp(-|b|^2/c).

    Taylor-normalised arrays (entry alpha divided by alpha1! alpha2!) turn the
    two-variable Leibniz rule into a truncated two-dimensional convolution;
    D^gamma E = e1[gamma1] e2[gamma2] factorises per axis, so the convolution is
    evaluated as two nested one-dimensional sums (lower-triangular Toeplitz
    products) per pair.
    """
    npair = s.shape[0]
    z = s[:, 0] + 1j * s[:, 1]
    fact = np.array([math.factorial(n) for n in range(P + 1)], dtype=np.float64)
    ar = np.arange(P + 1)
    A1, A2 = np.meshgrid(ar, ar, indexing="ij")
    inside = (A1 + A2) <= P
    # g_n = (-i/2pi) (-1)^n n! / z^{n+1};  D^a (V1 - i V2)_pv = i^{a2} g_{|a|}
    g = (-1j / (2.0 * math.pi)) * ((-1.0) ** ar * fact)[None, :] / z[:, None] ** (ar[None, :] + 1)
    nidx = np.where(inside, A1 + A2, 0)
    v = g[:, nidx] * ((1j) ** A2)[None] * inside[None]
    tay = 1.0 / (fact[:, None] * fact[None, :])
    pv1 = v.real * tay[None]
    pv2 = -v.imag * tay[None]
    x = (s[:, 0] ** 2 + s[:, 1] ** 2) / c
    tail = x < X_NO_TAIL
    if np.any(tail):
        rc = math.sqrt(c)
        ii = np.nonzero(tail)[0]
        ex1 = np.exp(-(s[ii, 0] / rc) ** 2)
        ex2 = np.exp(-(s[ii, 1] / rc) ** 2)
        # e_d[k] = c^{-k/2} d^k/dt^k exp(-t^2) / k! at t = b_d / sqrt(c)
        sc = ((-1.0) ** ar * c ** (-ar / 2.0) / fact)[None, :]
        e1 = _hermite(P, s[ii, 0] / rc) * ex1[:, None] * sc
        e2 = _hermite(P, s[ii, 1] / rc) * ex2[:, None] * sc
        toe = np.clip(A1 - A2, 0, None)
        low = (A1 >= A2)[None]
        T1 = e1[:, toe] * low          # T1[p, a1, b1] = e1[a1 - b1]
        T2 = e2[:, toe] * low          # T2[p, a2, b2] = e2[a2 - b2]
        for pv in (pv1, pv2):
            inner = np.matmul(pv[ii], np.swapaxes(T2, 1, 2))   # [b1, a2]
            corr = np.matmul(T1, inner)                        # [a1, a2]
            pv[ii] -= corr * inside[None]
    mi = multi_indices(P)
    J1 = np.empty((npair, len(mi)))
    J2 = np.empty((npair, len(mi)))
    for col, (a1, a2) in enumerate(mi):
        f = fact[a1] * fact[a2]
        J1[:, col] = pv1[:, a1, a2] * f
        J2[:, col] = pv2[:, a1, a2] * f
    return J1, J2


def pair_jet(s: np.ndarray, P: int, lam: float):
    """H^B_1, H^B_2 at separations s for all |alpha| <= P.

    s: (npairs, 2) separations (physical units).  Returns (J1, J2), each
    (npairs, (P+1)(P+2)/2) in column order (grouped by |alpha|, then alpha_2).
    """
    s = np.atleast_2d(np.asarray(s, dtype=np.float64))
    c = 2.0 * lam * lam
    x = (s[:, 0] ** 2 + s[:, 1] ** 2) / c
    nc = (P + 1) * (P + 2) // 2
    J1 = np.empty((s.shape[0], nc))
    J2 = np.empty((s.shape[0], nc))
    x_split = max(2.5, 0.3 * P)
    for mask, fn in ((x < x_split, _near), (x >= x_split, _far)):
        sel = np.nonzero(mask)[0]
        for start in range(0, sel.size, _CHUNK):
            ii = sel[start:start + _CHUNK]
            a, b = fn(s[ii], P, c)
            J1[ii] = a
            J2[ii] = b
    return J1, J2
