"""Pins of the oracle on the coarse-grid tripole (Section 3.2.2) against the
paper's Table 1 (Section 4.2, tests/golden/table1_tripole_errors.txt).

A 6 x 6 grid of Gaussian vortices (eq:blurredIC) approximates the perturbed
Lamb-Oseen vortex of eq:perturbM2; the grid is run with m = 0 (a core
spreading vortex method) and with m = 2, and both are compared with one
particle carrying the expansion of the same initial field at high order.

What the paper's table fixes, and what is checked here at t = 1 and 2 (the
full table to t = 16 with the order-24 reference runs on the GPU):
* m = 2 is about 4 times more accurate than m = 0 early on (Table 1: 3.7x
  in L2 at t = 1 and 2);
* the errors grow linearly at first (Table 1: e(2) / e(1) = 1.98);
* the magnitudes agree with Table 1 within a factor 2.5.  The paper does not
  state where the grid's nodes sit, their areas or the sampling of the
  norms; with the readings taken here (nodes on the end points, area h^2,
  a uniform grid on [-6, 6]^2) the errors come out at 0.58 of the table's.
"""
import math
from pathlib import Path

import numpy as np
import pytest

import mmvm_inputs
from oracle.diagnostics import relative_errors, shifted_gaussians_expansion, vorticity
from oracle.integrate import dopri5
from oracle.rhs import lam_at

GOLDEN = Path(__file__).parent / "golden" / "table1_tripole_errors.txt"


def table1():
    rows = [r.split() for r in GOLDEN.read_text().splitlines() if r and not r.startswith("#")]
    return {int(r[0]): tuple(float(v) for v in r[1:]) for r in rows}


def _grid(half=6.0, npt=121):
    g = np.linspace(-half, half, npt)
    P1, P2 = np.meshgrid(g, g, indexing="ij")
    return np.stack([P1.ravel(), P2.ravel()], axis=1)


def test_single_particle_expansion_reproduces_the_gaussians():
    """Taylor's theorem in the shift: the order-16 single-particle moments
    rebuild the field of the 36 Gaussians (their largest shift is sqrt(2)
    core sizes, so the remainder is below 1e-4)."""
    wl = mmvm_inputs.tripole_coarse_grid(order=0)
    pts = _grid(4.0, 81)
    exact = vorticity(wl.x, wl.moments, wl.lam0, 0, pts)
    ref = shifted_gaussians_expansion(wl.x, wl.moments[:, 0], 16)
    approx = vorticity(np.zeros((1, 2)), ref, wl.lam0, 16, pts)
    assert relative_errors(approx, exact)[0] < 1e-4
    # a single Gaussian at a: M_k = (-a)^k / k! exactly
    one = shifted_gaussians_expansion(np.array([[0.3, -0.5]]), np.array([2.0]), 3)
    assert one[0, 1] == pytest.approx(-0.6) and one[0, 2] == pytest.approx(1.0)
    assert one[0, 3] == pytest.approx(2.0 * 0.09 / 2) and one[0, 4] == pytest.approx(2.0 * -0.3 * 0.5)


def test_early_errors_match_table_1():
    ref_order = 12
    pts = _grid()
    paper = table1()
    runs = {}
    for m in (0, 2):
        wl = mmvm_inputs.tripole_coarse_grid(order=m)
        runs[m] = (wl.x, wl.moments, m)
    wl0 = mmvm_inputs.tripole_coarse_grid(order=0)
    runs["ref"] = (np.zeros((1, 2)), shifted_gaussians_expansion(wl0.x, wl0.moments[:, 0],
                                                                  ref_order), ref_order)
    lam0, nu = wl0.lam0, wl0.nu
    t = 0.0
    errs = {}
    for T in (1, 2):
        fields = {}
        for k, (x, mom, order) in runs.items():
            x, mom, tt, _, _ = dopri5(x, mom, t, float(T), 0.01, order, lam0, nu,
                                      rtol=1e-8, atol=1e-8)
            assert tt == T
            runs[k] = (x, mom, order)
            fields[k] = vorticity(x, mom, lam_at(T, lam0, nu), order, pts)
        t = float(T)
        errs[T] = {m: relative_errors(fields[m], fields["ref"]) for m in (0, 2)}
    for T in (1, 2):
        e0, e2 = errs[T][0], errs[T][2]
        assert 2.5 < e0[0] / e2[0] < 5.0  # L2: Table 1 3.7
        assert 2.0 < e0[1] / e2[1] < 5.0  # L-infinity: Table 1 3.9-4.0
        for got, want in zip((e0[0], e2[0], e0[1], e2[1]), paper[T]):
            assert want / 2.5 < got < want * 2.5
    for m in (0, 2):
        assert 1.7 < errs[2][m][0] / errs[1][m][0] < 2.3  # linear growth
    assert math.isfinite(errs[2][2][0])
