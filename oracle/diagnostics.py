"""Diagnostics of an MMVM state (oracle, FP64): the reconstructed vorticity
and the nonaxisymmetric enstrophy.

Test infrastructure only (see ``oracle/__init__.py``).

* Vorticity (eq:vorticity_decomposition, eq:moment_expansion_def_tw0):
      omega(x) = sum_j sum_{|k| <= M} M^j_k D^k phi_00(x - x^j; lambda),
      phi_00(x; lambda) = exp(-|x|^2 / lambda^2) / (pi lambda^2),
  and with t = x / lambda and the physicists' Hermite polynomials H_n
  (d^n/dt^n e^{-t^2} = (-1)^n H_n(t) e^{-t^2}):
      D^k phi_00(x) = (-1)^{|k|} lambda^{-|k|} H_{k1}(t1) H_{k2}(t2)
                      exp(-|t|^2) / (pi lambda^2).
* Nonaxisymmetric enstrophy (eq:nonaxi_enstrophy):
      E = int (omega(x) - <omega>(|x - c|))^2 dx,
      <omega>(r) = (1/2pi) int_0^{2pi} omega(c + r e_theta) dtheta,
  about a centre c, on a polar grid: the trapezoid rule in theta (spectrally
  accurate for a periodic integrand) and Gauss-Legendre in r on [0, r_max].
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import hermite as _herm

from .coefficients import multi_indices


def vorticity(x: np.ndarray, moments: np.ndarray, lam: float, order: int,
              pts: np.ndarray) -> np.ndarray:
    """omega at the points pts (npts, 2) of the state (x, moments) at core lam."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    moments = np.atleast_2d(np.asarray(moments, dtype=np.float64))
    pts = np.atleast_2d(np.asarray(pts, dtype=np.float64))
    out = np.zeros(pts.shape[0])
    mi = multi_indices(order)
    eye = np.eye(order + 1)
    for j in range(x.shape[0]):
        t = (pts - x[j]) / lam
        g = np.exp(-(t[:, 0] ** 2 + t[:, 1] ** 2)) / (math.pi * lam * lam)
        H1 = np.stack([_herm.hermval(t[:, 0], eye[n]) for n in range(order + 1)])
        H2 = np.stack([_herm.hermval(t[:, 1], eye[n]) for n in range(order + 1)])
        acc = np.zeros(pts.shape[0])
        for col, (k1, k2) in enumerate(mi):
            mk = moments[j, col]
            if mk == 0.0:
                continue
            acc += mk * (-1.0) ** (k1 + k2) * lam ** (-(k1 + k2)) * H1[k1] * H2[k2]
        out += acc * g
    return out


def polar_grid(cx: float, cy: float, r_max: float, nr: int, ntheta: int):
    """Nodes (nr * ntheta, 2) and weights of the polar quadrature: Gauss-
    Legendre in r on [0, r_max] (weight r dr), trapezoid in theta."""
    xg, wg = np.polynomial.legendre.leggauss(nr)
    r = 0.5 * r_max * (xg + 1.0)
    wr = 0.5 * r_max * wg * r
    th = 2.0 * math.pi * np.arange(ntheta) / ntheta
    R, TH = np.meshgrid(r, th, indexing="ij")
    pts = np.stack([cx + R.ravel() * np.cos(TH.ravel()), cy + R.ravel() * np.sin(TH.ravel())],
                   axis=1)
    return pts, r, wr, 2.0 * math.pi / ntheta


def nonaxi_enstrophy(x, moments, lam, order, cx=0.0, cy=0.0, r_max=None, nr=96,
                     ntheta=128) -> float:
    """E of eq:nonaxi_enstrophy about (cx, cy) on the polar grid above."""
    if r_max is None:
        spread = np.abs(np.atleast_2d(x) - np.array([cx, cy])).max() if np.size(x) else 0.0
        r_max = spread + 9.0 * lam
    pts, r, wr, dth = polar_grid(cx, cy, r_max, nr, ntheta)
    w = vorticity(x, moments, lam, order, pts).reshape(nr, ntheta)
    dev = w - w.mean(axis=1, keepdims=True)
    return float(np.sum(wr * (dev ** 2).sum(axis=1)) * dth)
