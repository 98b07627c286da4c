"""The allocation-free right-hand side (mmvm_rhs_noalloc) against the context
entry point (mmvm_rhs_device) on the same inputs, through the C ABI.

Both run the same kernels; they differ in where the scratch lives (a fixed
device array vs buffers the context allocates) and in how the sources are
split into chunks, so they agree to rounding: the FP64 and mixed-precision
tolerances are those of the GPU parity tests.  Each case calls the
allocation-free entry point twice in a row: the second call reuses the
scratch the first one left behind.  This file runs last (its name sorts
last) and also passes alone in a fresh process.
"""
import numpy as np
import pytest

import mmvm_inputs
from tests.parity_util import rhs_error, vel_error
from tests.test_gpu_parity import FP64_TOL, MIXED_RHS_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_1010_2475_gb300 as mm

    mm.load_library()
    torch.cuda.set_device(0)
    return torch, mm


def _context_rhs(mm, wl, t, prec):
    flags = mm.MMVM_FLAG_NO_FAR_FIELD  # the allocation-free path has no far field
    with mm.Context(wl.order, wl.lam0, wl.nu, prec, flags=flags) as ctx:
        ctx.set_state(wl.x, wl.moments, t)
        return ctx.rhs()


def _noalloc_rhs(torch, mm, wl, t, prec):
    dev = torch.device("cuda", 0)
    d_x = torch.from_numpy(np.ascontiguousarray(wl.x)).to(dev)
    d_m = torch.from_numpy(np.ascontiguousarray(wl.moments)).to(dev)
    d_dx = torch.full((wl.n, 2), float("nan"), dtype=torch.float64, device=dev)
    d_dm = torch.full((wl.n, wl.K), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    mm.mmvm_rhs_noalloc(wl.order, wl.lam0, wl.nu, prec, wl.n, t, d_x.data_ptr(),
                        d_m.data_ptr(), d_dx.data_ptr(), d_dm.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return d_dx.cpu().numpy(), d_dm.cpu().numpy()


def _check(gx, gM, rx, rM, wl, t, tol):
    from oracle.rhs import lam_at

    assert np.all(np.isfinite(gx)) and np.all(np.isfinite(gM))
    if wl.n == 1:  # a lone particle does not move (no other particle induces a velocity)
        assert np.all(gx == 0.0) and np.all(rx == 0.0)
    else:
        assert vel_error(gx, rx) <= tol
    if wl.order >= 2:
        assert rhs_error(gM, rM, wl.order, lam_at(t, wl.lam0, wl.nu)) <= tol


CASES = [
    # (order, n, precision): several CTA tiles with a ragged tail, two source
    # chunks, the largest n the fixed scratch takes, and a single particle
    (4, 600, "mixed"),
    (4, 600, "fp64"),
    (6, 333, "mixed"),
    (2, 4096, "mixed"),
    (8, 129, "fp64"),
    (8, 1, "fp64"),
]


@pytest.mark.parametrize("order,n,prec", CASES)
def test_noalloc_matches_context_twice(env, order, n, prec):
    torch, mm = env
    wl = mmvm_inputs.random_disk(n=n, order=order, radius=2.0 + 0.15 * n ** 0.5, sigma=0.45,
                                 amp=0.03, moment_scale="absolute", seed=700 + order)
    if n == 1:
        wl = mmvm_inputs.single_quadrupole(order=order, eps=0.1, sigma0=1.0)
    t = 0.4
    p = mm.MMVM_FP64 if prec == "fp64" else mm.MMVM_MIXED_FP32
    tol = FP64_TOL if prec == "fp64" else MIXED_RHS_TOL
    rx, rM = _context_rhs(mm, wl, t, p)
    for _ in range(2):  # two calls in a row share the scratch
        gx, gM = _noalloc_rhs(torch, mm, wl, t, p)
        _check(gx, gM, rx, rM, wl, t, tol)


def test_noalloc_alternating_orders(env):
    """Calls that switch order re-upload the tables; results stay right."""
    torch, mm = env
    a = mmvm_inputs.random_disk(n=300, order=3, radius=3.0, sigma=0.45, amp=0.03, moment_scale="absolute", seed=801)
    b = mmvm_inputs.random_disk(n=200, order=5, radius=3.0, sigma=0.45, amp=0.03, moment_scale="absolute", seed=802)
    refs = {id(w): _context_rhs(mm, w, 0.2, mm.MMVM_FP64) for w in (a, b)}
    for w in (a, b, a):
        gx, gM = _noalloc_rhs(torch, mm, w, 0.2, mm.MMVM_FP64)
        _check(gx, gM, *refs[id(w)], w, 0.2, FP64_TOL)


def test_noalloc_rejects_sizes_beyond_the_scratch(env):
    torch, mm = env
    dev = torch.device("cuda", 0)
    buf = torch.zeros(16, dtype=torch.float64, device=dev)
    p = buf.data_ptr()
    with pytest.raises(mm.MMVMError) as ei:
        mm.mmvm_rhs_noalloc(4, 0.5, 1e-3, mm.MMVM_FP64, 4097, 0.0, p, p, p, p)
    assert ei.value.code == mm.MMVM_E_UNSUPPORTED
    assert "4096" in str(ei.value)
    with pytest.raises(mm.MMVMError) as ei:
        mm.mmvm_rhs_noalloc(9, 0.5, 1e-3, mm.MMVM_FP64, 10, 0.0, p, p, p, p)
    assert ei.value.code == mm.MMVM_E_UNSUPPORTED
