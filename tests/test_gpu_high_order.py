"""Single particle at high order: the separable self-term path of the CUDA
library (used above order 16, forced below it by MMVM_FLAG_SEPARABLE_SELF)
against the oracle's rows (oracle.rhs.self_rhs_rows) and against the table
path.

Tolerance: per moment row, |dM_k(GPU) - dM_k(oracle)| <= 64 eps S_k, with S_k
the sum of the absolute values of the row's terms (both evaluations round
every term to a relative eps; 64 covers the accumulated rounding of either
summation order).  A row without terms must come out exactly zero.
"""
import numpy as np
import pytest

import mmvm_inputs
from oracle.coefficients import multi_indices
from oracle.rhs import lam_at, self_rhs_rows

pytestmark = pytest.mark.gpu

EPS = 2.220446049250313e-16


@pytest.fixture(scope="module")
def mm():
    import paper_1010_2475_gb300 as mm

    mm.load_library()
    return mm


def _gpu_rhs(mm, wl, t, flags=0):
    with mm.Context(wl.order, wl.lam0, wl.nu, mm.MMVM_FP64, flags=flags) as ctx:
        ctx.set_state(wl.x, wl.moments, t)
        return ctx.rhs()


def _check_rows(gM, wl, t, rows):
    lam = lam_at(t, wl.lam0, wl.nu)
    v, a = self_rhs_rows(wl.moments[0], lam, wl.order, rows)
    d = np.abs(gM[0, rows] - v)
    assert np.all(d <= 64 * EPS * a), (d / np.where(a > 0, a, 1)).max()


def _weighted_state(order, seed, sigma=0.8, amp=0.05):
    return mmvm_inputs.random_disk(n=1, order=order, radius=0.0, sigma=sigma, amp=amp, Re=700.0,
                                   seed=seed)


@pytest.mark.parametrize("order", [0, 2, 5, 8, 12, 16])
def test_separable_path_matches_oracle_and_tables(mm, order):
    wl = _weighted_state(order, 60 + order)
    t = 0.3
    gx_s, gM_s = _gpu_rhs(mm, wl, t, flags=mm.MMVM_FLAG_SEPARABLE_SELF)
    gx_t, gM_t = _gpu_rhs(mm, wl, t)
    assert np.all(gx_s == 0.0) and np.all(gx_t == 0.0)
    rows = list(range(wl.K))
    _check_rows(gM_s, wl, t, rows)
    _check_rows(gM_t, wl, t, rows)


def test_order_60_quadrupole(mm):
    """The high-order single-particle configuration: Lamb-Oseen core plus a
    quadrupole of amplitude 0.1 on (2,0)/(0,2)/(1,1), order 60 (1891 moments)."""
    wl = mmvm_inputs.single_quadrupole(order=60, eps=0.1, sigma0=1.0, Re=1000.0, dt=0.01)
    t = 0.5
    gx, gM = _gpu_rhs(mm, wl, t)
    assert np.all(np.isfinite(gM)) and np.all(gx == 0.0)
    rng = np.random.default_rng(0)
    rows = sorted(set(range(21)) | set(rng.integers(21, wl.K, 20).tolist()))
    _check_rows(gM, wl, t, rows)


def test_order_60_dense_state(mm):
    """Every one of the 1891 moments nonzero (1% per moment in the weighted
    norm), so every term of every row is present."""
    wl = _weighted_state(60, 61, sigma=1.0, amp=0.01)
    t = 0.2
    gx, gM = _gpu_rhs(mm, wl, t)
    rng = np.random.default_rng(1)
    mi = multi_indices(60)
    rows = sorted(set(rng.integers(0, wl.K, 14).tolist())
                  | {mi.index((1, 1)), mi.index((30, 30)), mi.index((59, 1)), mi.index((0, 60))})
    _check_rows(gM, wl, t, rows)


def test_order_60_dense_state_against_exact_rows(mm):
    """The dense order-60 state at t = 0 (lambda = 1) against the exact
    rational rows of tests/golden/order60_dense_exact.txt (oracle/exact.py):
    every row within 64 eps of its absolute term sum S_k, and within 1e-6 of
    the row itself where its condition number S_k / |dM_k| is below 1e8.
    The second bound fails for a GPU row off by more than rounding on the
    rows FP64 can resolve; the first is all FP64 promises on the rest (their
    condition numbers reach 1e26)."""
    import os

    from tests.golden.make_order60_exact import dense_state, rows

    g = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "order60_dense_exact.txt"))
    wl = dense_state()
    gx, gM = _gpu_rhs(mm, wl, 0.0)
    v = gM[0, rows()]
    d = np.abs(v - g[:, 2])
    assert np.all(d <= 64 * EPS * g[:, 3]), (d / g[:, 3]).max()
    good = g[:, 3] < 1e8 * np.abs(g[:, 2])
    assert good.sum() >= 3
    assert np.all(d[good] <= 1e-6 * np.abs(g[good, 2])), (d[good] / np.abs(g[good, 2])).max()


def test_order_60_steps_keep_the_invariants(mm):
    """RK4 at order 60: the circulation M_00 never changes (its row has no
    term), the centre stays put, the first moments stay zero."""
    wl = mmvm_inputs.single_quadrupole(order=60, eps=0.1, sigma0=1.0, Re=1000.0, dt=0.01)
    with mm.Context(wl.order, wl.lam0, wl.nu, mm.MMVM_FP64) as ctx:
        ctx.set_state(wl.x, wl.moments, 0.0)
        ctx.step(wl.dt, 50)
        x, m, t = ctx.get_state()
    assert abs(t - 0.5) < 1e-12
    assert np.all(x == 0.0)
    assert m[0, 0] == wl.moments[0, 0]
    assert np.all(m[0, 1:3] == 0.0)
    assert np.all(np.isfinite(m))
    assert np.abs(m[0, 3:6] - wl.moments[0, 3:6]).max() > 1e-6  # the quadrupole did evolve


def test_separable_and_table_trajectories_agree(mm):
    """Twenty RK4 steps at order 12 by both routes agree to rounding (1e-10
    relative in the weighted norm)."""
    wl = _weighted_state(12, 70)
    out = []
    for flags in (0, mm.MMVM_FLAG_SEPARABLE_SELF):
        with mm.Context(wl.order, wl.lam0, wl.nu, mm.MMVM_FP64, flags=flags) as ctx:
            ctx.set_state(wl.x, wl.moments, 0.0)
            ctx.step(0.01, 20)
            out.append(ctx.get_state()[1])
    from tests.parity_util import state_error

    assert state_error(out[1], out[0], 12, lam_at(0.2, wl.lam0, wl.nu)) <= 1e-10


def test_separable_flag_needs_one_particle(mm):
    wl = mmvm_inputs.random_disk(n=4, order=4, radius=2.0, sigma=0.5, seed=3)
    with mm.Context(4, wl.lam0, wl.nu, mm.MMVM_FP64, flags=mm.MMVM_FLAG_SEPARABLE_SELF) as ctx:
        with pytest.raises(mm.MMVMError) as ei:
            ctx.set_state(wl.x, wl.moments, 0.0)
        assert ei.value.code == mm.MMVM_E_UNSUPPORTED
