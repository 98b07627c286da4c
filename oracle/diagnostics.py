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
* The single-particle expansion of a set of Gaussian vortices (the reference
  of the coarse-grid tripole, Section 3.2.2) and the relative L2 / L-infinity
  errors of a sampled vorticity field (Section 4.2, Table 1).
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


def shifted_gaussians_expansion(x: np.ndarray, m00: np.ndarray, order: int,
                                centre=(0.0, 0.0)) -> np.ndarray:
    """Moments (1, K) about `centre` of the field sum_j m00_j phi_00(p - x^j)
    in the basis D^k phi_00 of the same core (the single-particle form of a
    set of Gaussian vortices, as the order-24 reference of Section 3.2.2
    uses).  Taylor's theorem in the shift a_j = x^j - centre gives, for every
    core, phi_00(p - a) = sum_k (-a)^k / k! D^k phi_00(p), so
        M_k = sum_j m00_j (-a_j1)^k1 (-a_j2)^k2 / (k1! k2!),
    exact up to the truncation at total order `order`."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    a = x - np.asarray(centre, dtype=np.float64)
    m00 = np.asarray(m00, dtype=np.float64).ravel()
    mi = multi_indices(order)
    out = np.zeros((1, len(mi)))
    for col, (k1, k2) in enumerate(mi):
        out[0, col] = np.sum(m00 * (-a[:, 0]) ** k1 * (-a[:, 1]) ** k2) / (
            math.factorial(k1) * math.factorial(k2))
    return out


def relative_errors(w: np.ndarray, w_ref: np.ndarray) -> tuple:
    """(relative L2, relative L-infinity) error of the sampled field w against
    w_ref on the same uniform grid (Section 4.2): ||w - w_ref|| / ||w_ref||."""
    d = np.asarray(w) - np.asarray(w_ref)
    return (float(np.linalg.norm(d) / np.linalg.norm(w_ref)),
            float(np.abs(d).max() / np.abs(w_ref).max()))
