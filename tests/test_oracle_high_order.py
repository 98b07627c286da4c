"""Pins of the oracle's single-particle rows (oracle.rhs.self_rhs_rows) up to
order 60, where the full term list no longer fits.

* Every row equals the full regrouped evaluation (rhs_regrouped, itself
  pinned by quadrature and the invariants) at orders 6 and 10.
* P-1/P-2 at M = 60: the Lamb-Oseen core-mismatch state of Section 4.1.1
  (mu_0 = 2.1 at lambda_0 = 2) and a radial state with random radial
  coefficients are steady, so every sampled row vanishes to rounding of its
  own terms.
* P-3/P-6: dM_00 has no term at all; for a state with even-even moments
  only, every row except those with k1 and k2 both odd vanishes term by term
  (the parity rule: H_1(a) needs a1 even and a2 odd, H_2(a) the reverse, so a
  term needs k1 + l1 + m1 and k2 + l2 + m2 both odd).
"""
import math

import numpy as np
import pytest

import mmvm_inputs
from oracle.coefficients import idx, multi_indices, n_moments
from oracle.rhs import rhs_regrouped, self_rhs_rows

EPS = 2.220446049250313e-16


@pytest.mark.parametrize("order", [6, 10])
def test_rows_equal_the_full_evaluation(order):
    wl = mmvm_inputs.random_disk(n=1, order=order, radius=0.0, sigma=0.8, amp=0.05, seed=order)
    dx, dM = rhs_regrouped(wl.x, wl.moments, 0.0, order, wl.lam0, 0.0)
    v, a = self_rhs_rows(wl.moments[0], wl.lam0, order, range(wl.K))
    assert np.all(np.abs(v - dM[0]) <= 16 * EPS * a)


def _radial_state(order, g):
    mom = np.zeros(n_moments(order))
    for a in range(order // 2 + 1):
        for b in range(order // 2 + 1 - a):
            mom[idx(2 * a, 2 * b)] = g[a + b] * math.comb(a + b, a)
    return mom


def _sample_rows(order, count, seed):
    """Rows with k1 and k2 both odd (the rows that carry terms for a state of
    even-even moments), low, middle and highest orders among them."""
    rng = np.random.default_rng(seed)
    mi = multi_indices(order)
    both_odd = [c for c, (k1, k2) in enumerate(mi) if k1 % 2 == 1 and k2 % 2 == 1]
    rows = set(rng.choice(both_odd, size=count, replace=False).tolist())
    h = order // 2 - 1 if (order // 2) % 2 == 0 else order // 2
    top = order - 1 if (order - 1) % 2 == 1 else order - 2
    rows |= {idx(1, 1), idx(3, 1), idx(h, h), idx(top, 1)}
    return sorted(rows)


def test_lamb_oseen_mismatch_is_steady_at_order_60():
    order, lam0, mu0 = 60, 2.0, 2.1
    d = mu0 ** 2 - lam0 ** 2
    g = [(d / 4) ** n / math.factorial(n) for n in range(order // 2 + 1)]
    mom = _radial_state(order, g)
    rows = _sample_rows(order, 6, 1)
    v, a = self_rhs_rows(mom, lam0, order, rows)
    assert np.all(a > 0)
    assert np.all(np.abs(v) <= 64 * EPS * a)


def test_random_radial_state_is_steady_at_order_60():
    order = 60
    rng = np.random.default_rng(3)
    g = [rng.normal() * 0.6 ** n / math.sqrt(math.factorial(n)) for n in range(order // 2 + 1)]
    mom = _radial_state(order, g)
    rows = _sample_rows(order, 6, 2)
    v, a = self_rhs_rows(mom, 1.3, order, rows)
    assert np.all(a > 0)
    assert np.all(np.abs(v) <= 64 * EPS * a)


def test_circulation_row_and_parity_rule():
    order = 20
    wl = mmvm_inputs.single_quadrupole(order=order, eps=0.1, sigma0=1.0, with_11=False)
    mi = multi_indices(order)
    other = [c for c, (k1, k2) in enumerate(mi) if not (k1 % 2 == 1 and k2 % 2 == 1)]
    v, a = self_rhs_rows(wl.moments[0], 1.0, order, other)
    assert v[0] == 0.0 and a[0] == 0.0  # no term of eq:FinalSingleI/II for k = 0
    assert np.all(v == 0.0) and np.all(a == 0.0)
    # the quadrupole does evolve: (2,0) - (0,2) turns into (1,1) (rotation)
    v2, a2 = self_rhs_rows(wl.moments[0], 1.0, order, [idx(1, 1), idx(3, 1)])
    assert np.all(a2 > 0) and abs(v2[0]) > 1e-3


def test_exact_rows_match_fp64_rows_at_low_order():
    """oracle/exact.py (rational arithmetic, one rounding at the end) against
    the FP64 rows of self_rhs_rows on every row of a dense order-8 state at
    lambda = 1: the two agree to the FP64 rounding of the row's terms."""
    import mmvm_inputs
    from oracle.exact import self_rows_exact, to_float
    from oracle.rhs import self_rhs_rows

    wl = mmvm_inputs.random_disk(n=1, order=8, radius=0.0, sigma=1.0, amp=0.05, seed=8)
    rows = list(range(wl.K))
    v, a = self_rows_exact(wl.moments[0], 8, rows)
    ov, oa = self_rhs_rows(wl.moments[0], 1.0, 8, rows)
    ev = np.array([to_float(x) for x in v])
    ea = np.array([to_float(x) for x in a])
    assert np.all(np.abs(ov - ev) <= 8 * 2.220446049250313e-16 * ea)
    assert np.allclose(oa, ea, rtol=1e-13, atol=0.0)


def test_order60_dense_rows_against_exact():
    """The FP64 oracle at order 60 on a dense state (every one of the 1891
    moments nonzero) against the exact rational rows of
    tests/golden/order60_dense_exact.txt (written by make_order60_exact.py):
    within 4 eps of each row's absolute term sum S_k, and within 1e-10 of
    the row itself where the row's condition number S_k / |dM_k| is below
    1e8 (the golden rows reach condition numbers of 1e26, where no FP64
    evaluation can resolve the row at all)."""
    import os

    from tests.golden.make_order60_exact import dense_state, rows
    from oracle.rhs import self_rhs_rows

    g = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "order60_dense_exact.txt"))
    wl = dense_state()
    rr = rows()
    v, a = self_rhs_rows(wl.moments[0], 1.0, 60, rr)
    d = np.abs(v - g[:, 2])
    assert np.all(d <= 4 * 2.220446049250313e-16 * g[:, 3])
    good = g[:, 3] < 1e8 * np.abs(g[:, 2])
    assert good.sum() >= 3
    assert np.all(d[good] <= 1e-10 * np.abs(g[good, 2]))
    assert np.allclose(a, g[:, 3], rtol=1e-12, atol=0.0)
