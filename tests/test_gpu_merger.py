"""The two-vortex merger model (Section 3.2.1) on the GPU: adaptive
Dormand-Prince at 1e-8 (the paper's tolerance) through mmvm_integrate against
the oracle's dopri5 (same steps, 1e-9), mixed precision against FP64, and the
text's claims (m = 0 stays on the circle; merger regime falls and settles in
m; the well separated pair keeps its distance)."""
import math

import numpy as np
import pytest

import mmvm_inputs
from oracle.integrate import dopri5
from oracle.rhs import lam_at
from tests.parity_util import state_error

pytestmark = pytest.mark.gpu

T_STAR = (0.05, 0.1, 0.127, 0.152)


@pytest.fixture(scope="module")
def mm():
    import paper_1010_2475_gb300 as mm

    mm.load_library()
    return mm


def gpu_radii(mm, a_over_b, order, precision):
    wl = mmvm_inputs.vortex_pair(order=order, a_over_b=a_over_b)
    b = wl.meta["b"]
    out = []
    with mm.Context(order, wl.lam0, wl.nu, precision) as ctx:
        ctx.set_state(wl.x, wl.moments, 0.0)
        for ts in T_STAR:
            ctx.integrate(ts * 2 * math.pi ** 2 * b ** 2, h0=0.01, rtol=1e-8, atol=1e-8)
            x, mom, t = ctx.get_state()
            out.append((x, mom, t))
    return wl, out


@pytest.mark.parametrize("order", [0, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("a_over_b", [0.375, 0.125])
def test_fp64_matches_the_oracle(mm, a_over_b, order):
    wl, out = gpu_radii(mm, a_over_b, order, mm.MMVM_FP64)
    x, mom, t = wl.x, wl.moments, 0.0
    for ts, (gx, gm, gt) in zip(T_STAR, out):
        x, mom, t, _, _ = dopri5(x, mom, t, ts * 2 * math.pi ** 2 * wl.meta["b"] ** 2, 0.01,
                                 order, wl.lam0, wl.nu, rtol=1e-8, atol=1e-8)
        assert gt == t
        lam = lam_at(t, wl.lam0, wl.nu)
        assert np.abs(gx - x).max() <= 1e-9 * lam
        if order >= 2:
            assert state_error(gm, mom, order, lam) <= 1e-9


def test_claims_of_the_text(mm):
    r = {}
    for a_over_b in (0.375, 0.125):
        for order in (0, 2, 4, 5, 6):
            _, out = gpu_radii(mm, a_over_b, order, mm.MMVM_FP64)
            r[a_over_b, order] = np.array([np.linalg.norm(o[0][0]) for o in out])
    for a_over_b in (0.375, 0.125):
        assert np.abs(r[a_over_b, 0] - 1.0).max() < 1e-9
    assert 0.10 < 1.0 - r[0.375, 6][-1] < 0.30  # text: about 20 %
    assert np.abs(r[0.375, 6] - r[0.375, 5]).max() < 2e-3
    for order in (2, 4, 6):
        assert np.abs(r[0.125, order] - 1.0).max() < 0.01


@pytest.mark.parametrize("order", [2, 6])
def test_mixed_precision_follows_fp64(mm, order):
    wl, o64 = gpu_radii(mm, 0.375, order, mm.MMVM_FP64)
    _, o32 = gpu_radii(mm, 0.375, order, mm.MMVM_MIXED_FP32)
    for (x64, m64, t), (x32, m32, _) in zip(o64, o32):
        lam = lam_at(t, wl.lam0, wl.nu)
        assert np.abs(x32 - x64).max() <= 1e-5 * lam
        assert state_error(m32, m64, order, lam) <= 1e-5
