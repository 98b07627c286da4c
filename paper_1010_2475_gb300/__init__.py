"""Python binding of the GB300 MMVM library (libmmvm.so, C ABI in include/mmvm.h).

Argument marshalling only: every step of the right-hand side and of the RK4
integration runs in the library's CUDA kernels.  If libmmvm.so has not been
built (``python -m paper_1010_2475_gb300.build``) every call raises; there is
no CPU fallback.

The functions keep the C names (``mmvm_create``, ``mmvm_set_state``, ...).
Host arrays are float64 numpy arrays; the ``*_device`` variants take raw CUDA
pointers (for example ``torch.Tensor.data_ptr()`` of float64 CUDA tensors on
the context's device).  ``Context`` wraps a handle for convenience.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmmvm.so")

MMVM_OK = 0
MMVM_PENDING = 1
MMVM_E_INVALID_ARG = -1
MMVM_E_ZERO_CIRCULATION = -2
MMVM_E_UNSUPPORTED = -3
MMVM_E_OOM = -4
MMVM_E_NUMERIC = -5
MMVM_E_TIMEOUT = -6
MMVM_E_DEVICE = -7
MMVM_FP64 = 0
MMVM_MIXED_FP32 = 1
MMVM_FLAG_NO_FAR_FIELD = 1
MMVM_FLAG_SEPARABLE_SELF = 2
MMVM_MAX_ORDER_PAIRS = 8
MMVM_MAX_ORDER_SINGLE = 64

_ERRNAMES = {
    MMVM_E_INVALID_ARG: "INVALID_ARG",
    MMVM_E_ZERO_CIRCULATION: "ZERO_CIRCULATION",
    MMVM_E_UNSUPPORTED: "UNSUPPORTED",
    MMVM_E_OOM: "OOM",
    MMVM_E_NUMERIC: "NUMERIC",
    MMVM_E_TIMEOUT: "TIMEOUT",
    MMVM_E_DEVICE: "DEVICE",
}

# Every symbol include/mmvm.h declares (checked by the ABI test).
EXPORTS = (
    "mmvm_create", "mmvm_destroy", "mmvm_set_state", "mmvm_set_state_device",
    "mmvm_get_state", "mmvm_get_state_device", "mmvm_rhs", "mmvm_rhs_device",
    "mmvm_step", "mmvm_set_stream", "mmvm_synchronize", "mmvm_num_particles",
    "mmvm_num_moments", "mmvm_launch_count", "mmvm_last_error", "mmvm_last_error_string",
    "mmvm_enable_timing",
    "mmvm_pair_time", "mmvm_pair_time_parts", "mmvm_pair_config", "mmvm_pair_variant_counts",
    "mmvm_pair_counts",
    "mmvm_pair_work", "mmvm_alu_peak",
    "mmvm_rhs_noalloc", "mmvm_integrate", "mmvm_vorticity", "mmvm_nonaxi_enstrophy", "mmvm_server_create", "mmvm_server_destroy", "mmvm_submit",
    "mmvm_poll", "mmvm_server_stats", "mmvm_request_footprint",
)


class MMVMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class mmvm_config(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("lambda0", ctypes.c_double), ("nu", ctypes.c_double),
                ("device", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class mmvm_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_uint64), ("max_active", ctypes.c_int32),
                ("flags", ctypes.c_uint32)]


class mmvm_request(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("lambda0", ctypes.c_double),
                ("nu", ctypes.c_double), ("t0", ctypes.c_double), ("dt", ctypes.c_double),
                ("nsteps", ctypes.c_int64), ("n", ctypes.c_int64),
                ("x", ctypes.POINTER(ctypes.c_double)),
                ("moments", ctypes.POINTER(ctypes.c_double))]


class mmvm_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("order", ctypes.c_int32), ("n", ctypes.c_int64),
                ("steps_done", ctypes.c_int64), ("t", ctypes.c_double),
                ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]


class mmvm_server_counters(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("active", ctypes.c_int64), ("ticks", ctypes.c_int64),
                ("max_batch", ctypes.c_int64), ("max_active", ctypes.c_int64),
                ("pair_interactions", ctypes.c_double),
                ("busy_ms", ctypes.c_double), ("footprint_bytes", ctypes.c_uint64),
                ("peak_footprint_bytes", ctypes.c_uint64), ("budget_bytes", ctypes.c_uint64)]


_lib_handle = None


def load_library(path: str = LIB_PATH):
    """Load libmmvm.so (raises if it is missing: there is no fallback)."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_1010_2475_gb300.build` (CUDA toolkit needed)")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.POINTER(ctypes.c_double)
    lib.mmvm_create.argtypes = [ctypes.POINTER(mmvm_config), ctypes.POINTER(P)]
    lib.mmvm_create.restype = ctypes.c_int
    lib.mmvm_destroy.argtypes = [P]
    lib.mmvm_destroy.restype = None
    lib.mmvm_set_state.argtypes = [P, ctypes.c_int64, D, D, ctypes.c_double]
    lib.mmvm_set_state.restype = ctypes.c_int
    lib.mmvm_set_state_device.argtypes = [P, ctypes.c_int64, P, P, ctypes.c_double]
    lib.mmvm_set_state_device.restype = ctypes.c_int
    lib.mmvm_get_state.argtypes = [P, D, D, D]
    lib.mmvm_get_state.restype = ctypes.c_int
    lib.mmvm_get_state_device.argtypes = [P, P, P]
    lib.mmvm_get_state_device.restype = ctypes.c_int
    lib.mmvm_rhs.argtypes = [P, D, D]
    lib.mmvm_rhs.restype = ctypes.c_int
    lib.mmvm_rhs_device.argtypes = [P, P, P]
    lib.mmvm_rhs_device.restype = ctypes.c_int
    lib.mmvm_step.argtypes = [P, ctypes.c_double, ctypes.c_int64]
    lib.mmvm_step.restype = ctypes.c_int
    lib.mmvm_set_stream.argtypes = [P, P]
    lib.mmvm_set_stream.restype = ctypes.c_int
    lib.mmvm_synchronize.argtypes = [P]
    lib.mmvm_synchronize.restype = ctypes.c_int
    lib.mmvm_num_particles.argtypes = [P]
    lib.mmvm_num_particles.restype = ctypes.c_int64
    lib.mmvm_num_moments.argtypes = [ctypes.c_int32]
    lib.mmvm_num_moments.restype = ctypes.c_int32
    lib.mmvm_launch_count.argtypes = [P]
    lib.mmvm_launch_count.restype = ctypes.c_int64
    lib.mmvm_enable_timing.argtypes = [P, ctypes.c_int]
    lib.mmvm_enable_timing.restype = ctypes.c_int
    lib.mmvm_pair_time.argtypes = [P, D, ctypes.POINTER(ctypes.c_int64)]
    lib.mmvm_pair_time.restype = ctypes.c_int
    lib.mmvm_pair_time_parts.argtypes = [P, D, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int64)]
    lib.mmvm_pair_time_parts.restype = ctypes.c_int
    lib.mmvm_integrate.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int64,
                                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.mmvm_integrate.restype = ctypes.c_int
    lib.mmvm_vorticity.argtypes = [P, ctypes.c_int64, D, D]
    lib.mmvm_vorticity.restype = ctypes.c_int
    lib.mmvm_nonaxi_enstrophy.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int32, ctypes.c_int32, D]
    lib.mmvm_nonaxi_enstrophy.restype = ctypes.c_int
    lib.mmvm_rhs_noalloc.argtypes = [ctypes.POINTER(mmvm_config), ctypes.c_int64, ctypes.c_double,
                                     P, P, P, P, P]
    lib.mmvm_rhs_noalloc.restype = ctypes.c_int
    lib.mmvm_alu_peak.argtypes = [ctypes.c_int32, ctypes.c_int32,
                                  ctypes.POINTER(ctypes.c_double)]
    lib.mmvm_alu_peak.restype = ctypes.c_int
    lib.mmvm_pair_work.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    lib.mmvm_pair_work.restype = ctypes.c_int
    lib.mmvm_pair_counts.argtypes = [P, ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_int64)]
    lib.mmvm_pair_counts.restype = ctypes.c_int
    lib.mmvm_pair_config.argtypes = [P, ctypes.POINTER(ctypes.c_int32)]
    lib.mmvm_pair_config.restype = ctypes.c_int
    lib.mmvm_pair_variant_counts.argtypes = [ctypes.c_int32, ctypes.c_int32,
                                             ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_int32)]
    lib.mmvm_pair_variant_counts.restype = ctypes.c_int
    lib.mmvm_server_create.argtypes = [ctypes.POINTER(mmvm_server_config), ctypes.POINTER(P)]
    lib.mmvm_server_create.restype = ctypes.c_int
    lib.mmvm_server_destroy.argtypes = [P]
    lib.mmvm_server_destroy.restype = None
    lib.mmvm_submit.argtypes = [P, ctypes.POINTER(mmvm_request), ctypes.POINTER(ctypes.c_uint64)]
    lib.mmvm_submit.restype = ctypes.c_int
    lib.mmvm_poll.argtypes = [P, ctypes.c_uint64, D, D, ctypes.POINTER(mmvm_result)]
    lib.mmvm_poll.restype = ctypes.c_int
    lib.mmvm_server_stats.argtypes = [P, ctypes.POINTER(mmvm_server_counters)]
    lib.mmvm_server_stats.restype = ctypes.c_int
    lib.mmvm_request_footprint.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                           ctypes.POINTER(ctypes.c_uint64)]
    lib.mmvm_request_footprint.restype = ctypes.c_int
    lib.mmvm_last_error.argtypes = []
    lib.mmvm_last_error.restype = ctypes.c_char_p
    lib.mmvm_last_error_string.argtypes = []
    lib.mmvm_last_error_string.restype = ctypes.c_char_p
    _lib_handle = lib
    return lib


def _check(rc: int):
    if rc < 0:
        msg = load_library().mmvm_last_error()
        raise MMVMError(rc, msg.decode() if msg else "")
    return rc


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def n_moments(order: int) -> int:
    return (order + 1) * (order + 2) // 2


def mmvm_create(order: int, lambda0: float, nu: float, precision: int = MMVM_FP64,
                device: int = 0, flags: int = 0) -> ctypes.c_void_p:
    cfg = mmvm_config(order, precision, lambda0, nu, device, flags)
    h = ctypes.c_void_p()
    _check(load_library().mmvm_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def mmvm_destroy(h) -> None:
    load_library().mmvm_destroy(h)


def mmvm_set_state(h, x: np.ndarray, moments: np.ndarray, t: float) -> None:
    x = np.ascontiguousarray(x, dtype=np.float64)
    moments = np.ascontiguousarray(moments, dtype=np.float64)
    if x.ndim != 2 or x.shape[1] != 2 or moments.ndim != 2 or moments.shape[0] != x.shape[0]:
        raise ValueError("x must be (n, 2) and moments (n, K)")
    _check(load_library().mmvm_set_state(h, x.shape[0], _dptr(x), _dptr(moments), float(t)))


def mmvm_set_state_device(h, n: int, d_x: int, d_moments: int, t: float) -> None:
    _check(load_library().mmvm_set_state_device(h, n, ctypes.c_void_p(d_x),
                                                ctypes.c_void_p(d_moments), float(t)))


def mmvm_get_state(h, order: int):
    lib = load_library()
    n = lib.mmvm_num_particles(h)
    x = np.empty((n, 2))
    m = np.empty((n, n_moments(order)))
    t = ctypes.c_double()
    _check(lib.mmvm_get_state(h, _dptr(x), _dptr(m), ctypes.byref(t)))
    return x, m, t.value


def mmvm_get_state_device(h, d_x: int, d_moments: int) -> None:
    _check(load_library().mmvm_get_state_device(h, ctypes.c_void_p(d_x), ctypes.c_void_p(d_moments)))


def mmvm_rhs(h, order: int):
    lib = load_library()
    n = lib.mmvm_num_particles(h)
    dx = np.empty((n, 2))
    dm = np.empty((n, n_moments(order)))
    _check(lib.mmvm_rhs(h, _dptr(dx), _dptr(dm)))
    return dx, dm


def mmvm_rhs_device(h, d_dx: int, d_dm: int) -> None:
    _check(load_library().mmvm_rhs_device(h, ctypes.c_void_p(d_dx), ctypes.c_void_p(d_dm)))


def mmvm_step(h, dt: float, nsteps: int) -> None:
    _check(load_library().mmvm_step(h, float(dt), int(nsteps)))


def mmvm_set_stream(h, stream: Optional[int]) -> None:
    _check(load_library().mmvm_set_stream(h, ctypes.c_void_p(stream or 0)))


def mmvm_synchronize(h) -> None:
    _check(load_library().mmvm_synchronize(h))


def mmvm_launch_count(h) -> int:
    return int(load_library().mmvm_launch_count(h))


def mmvm_enable_timing(h, on: bool = True) -> None:
    _check(load_library().mmvm_enable_timing(h, 1 if on else 0))


def mmvm_pair_time(h):
    """(summed all-pairs device time in ms, number of launches) since the last call."""
    ms = ctypes.c_double()
    cnt = ctypes.c_int64()
    _check(load_library().mmvm_pair_time(h, ctypes.byref(ms), ctypes.byref(cnt)))
    return ms.value, cnt.value


def mmvm_pair_time_parts(h):
    """(per-kernel ms list of the list form: [list build + tree, far field,
    near kernels...], right-hand sides summed) since the previous call."""
    ms = (ctypes.c_double * 8)()
    npart = ctypes.c_int32()
    cnt = ctypes.c_int64()
    _check(load_library().mmvm_pair_time_parts(h, ms, 8, ctypes.byref(npart), ctypes.byref(cnt)))
    return list(ms)[:npart.value], cnt.value


def mmvm_integrate(h, t_end: float, h0: float = 0.01, rtol: float = 1e-8, atol: float = 1e-8,
                   max_steps: int = 1000000):
    """Adaptive Dormand-Prince 5(4) to t_end; returns (accepted, rejected) steps."""
    a = ctypes.c_int64()
    r = ctypes.c_int64()
    _check(load_library().mmvm_integrate(h, float(t_end), float(h0), float(rtol), float(atol),
                                         int(max_steps), ctypes.byref(a), ctypes.byref(r)))
    return a.value, r.value


def mmvm_vorticity(h, pts) -> np.ndarray:
    """Vorticity of the context's current state at the points pts (n, 2)."""
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 2)
    out = np.empty(pts.shape[0])
    _check(load_library().mmvm_vorticity(h, pts.shape[0], _dptr(pts), _dptr(out)))
    return out


def mmvm_nonaxi_enstrophy(h, cx: float, cy: float, r_max: float, nr: int = 96,
                          ntheta: int = 128) -> float:
    """Nonaxisymmetric enstrophy of the current state about (cx, cy)."""
    v = np.zeros(1)
    _check(load_library().mmvm_nonaxi_enstrophy(h, float(cx), float(cy), float(r_max), int(nr),
                                                 int(ntheta), _dptr(v)))
    return float(v[0])


def mmvm_rhs_noalloc(order: int, lambda0: float, nu: float, precision: int, n: int, t: float,
                     d_x: int, d_moments: int, d_dxdt: int, d_dMdt: int,
                     stream: int = 0) -> None:
    """Right-hand side from caller-owned device buffers, with no allocation
    (fixed scratch: n <= 4096, order <= 8); runs on the current device."""
    cfg = mmvm_config(order, precision, lambda0, nu, 0, 0)
    _check(load_library().mmvm_rhs_noalloc(
        ctypes.byref(cfg), int(n), float(t), ctypes.c_void_p(d_x), ctypes.c_void_p(d_moments),
        ctypes.c_void_p(d_dxdt), ctypes.c_void_p(d_dMdt), ctypes.c_void_p(stream)))


def mmvm_alu_peak(device: int = 0, precision: int = MMVM_MIXED_FP32) -> float:
    """Measured FMA peak of the device in flop/s (FP32 or FP64 pipe)."""
    v = ctypes.c_double()
    _check(load_library().mmvm_alu_peak(device, precision, ctypes.byref(v)))
    return v.value


def mmvm_pair_work(h):
    """(near pairs, far pairs source by source, tile expansions evaluated,
    pairs covered by tile expansions) of the all-pairs kernel so far."""
    out = (ctypes.c_int64 * 4)()
    _check(load_library().mmvm_pair_work(h, out))
    return tuple(int(v) for v in out)


def mmvm_pair_counts(h):
    """(near pairs, far pairs) evaluated by the all-pairs kernel so far."""
    a = ctypes.c_int64()
    b = ctypes.c_int64()
    _check(load_library().mmvm_pair_counts(h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def mmvm_pair_config(h) -> dict:
    """Variant of the all-pairs kernel in use (see include/mmvm.h)."""
    out = (ctypes.c_int32 * 8)()
    _check(load_library().mmvm_pair_config(h, out))
    return dict(zip(("variant", "order_slices", "targets_per_cta", "ctas_per_sm",
                     "sync", "chunks", "list_form", "far_ranges"), list(out)))


def pair_variant_counts(order: int, precision: int = MMVM_MIXED_FP32):
    """(direct-form variants, list-form variants) compiled for an order."""
    a = ctypes.c_int32()
    b = ctypes.c_int32()
    _check(load_library().mmvm_pair_variant_counts(order, precision, ctypes.byref(a),
                                                   ctypes.byref(b)))
    return a.value, b.value


class Context:
    """Owning wrapper of an mmvm_ctx handle."""

    def __init__(self, order: int, lambda0: float, nu: float, precision: int = MMVM_FP64,
                 device: int = 0, flags: int = 0):
        self.order = order
        self.handle = mmvm_create(order, lambda0, nu, precision, device, flags)

    def set_state(self, x, moments, t=0.0):
        mmvm_set_state(self.handle, x, moments, t)

    def get_state(self):
        return mmvm_get_state(self.handle, self.order)

    def rhs(self):
        return mmvm_rhs(self.handle, self.order)

    def integrate(self, t_end, h0=0.01, rtol=1e-8, atol=1e-8, max_steps=1000000):
        return mmvm_integrate(self.handle, t_end, h0, rtol, atol, max_steps)

    def vorticity(self, pts):
        return mmvm_vorticity(self.handle, pts)

    def nonaxi_enstrophy(self, cx=0.0, cy=0.0, r_max=10.0, nr=96, ntheta=128):
        return mmvm_nonaxi_enstrophy(self.handle, cx, cy, r_max, nr, ntheta)

    def step(self, dt, nsteps=1):
        mmvm_step(self.handle, dt, nsteps)

    def synchronize(self):
        mmvm_synchronize(self.handle)

    @property
    def launches(self) -> int:
        return mmvm_launch_count(self.handle)

    def close(self):
        if self.handle:
            mmvm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ------------------------------------------------------------------ serving
def mmvm_request_footprint(order: int, precision: int, n: int) -> int:
    """Device bytes a request holds while admitted (host-only computation)."""
    v = ctypes.c_uint64()
    _check(load_library().mmvm_request_footprint(order, precision, n, ctypes.byref(v)))
    return v.value


class Server:
    """Continuous-batching request loop (mmvm_server_*): submit simulations,
    poll for their final states."""

    def __init__(self, precision: int = MMVM_MIXED_FP32, device: int = 0,
                 hbm_budget_bytes: int = 0, max_active: int = 0, flags: int = 0):
        self.handle = ctypes.c_void_p()
        cfg = mmvm_server_config(device, precision, hbm_budget_bytes, max_active, flags)
        _check(load_library().mmvm_server_create(ctypes.byref(cfg), ctypes.byref(self.handle)))
        self._orders = {}

    def submit(self, x, moments, order: int, lambda0: float, nu: float, dt: float,
               nsteps: int, t0: float = 0.0) -> int:
        x = np.ascontiguousarray(x, dtype=np.float64)
        moments = np.ascontiguousarray(moments, dtype=np.float64)
        n = x.shape[0]
        if x.shape != (n, 2) or moments.shape != (n, (order + 1) * (order + 2) // 2):
            raise ValueError("x must be (n, 2) and moments (n, K)")
        req = mmvm_request(order, lambda0, nu, t0, dt, nsteps, n, _dptr(x), _dptr(moments))
        ticket = ctypes.c_uint64()
        _check(load_library().mmvm_submit(self.handle, ctypes.byref(req), ctypes.byref(ticket)))
        self._orders[ticket.value] = (order, n)
        return ticket.value

    def poll(self, ticket: int):
        """None while pending; else (x, moments, info dict)."""
        order, n = self._orders[ticket]
        K = (order + 1) * (order + 2) // 2
        x = np.empty((n, 2))
        m = np.empty((n, K))
        res = mmvm_result()
        rc = load_library().mmvm_poll(self.handle, ticket, _dptr(x), _dptr(m), ctypes.byref(res))
        if rc == MMVM_PENDING:
            return None
        del self._orders[ticket]
        info = {"t": res.t, "steps": res.steps_done, "queue_ms": res.queue_ms,
                "latency_ms": res.latency_ms}
        try:
            _check(rc)
        except MMVMError as e:  # the request failed; its timing is still known
            e.info = info
            raise
        return x, m, info

    def wait(self, ticket: int, timeout: float = 600.0, interval: float = 0.0005):
        import time

        t_end = time.monotonic() + timeout
        while True:
            r = self.poll(ticket)
            if r is not None:
                return r
            if time.monotonic() > t_end:
                raise TimeoutError(f"request {ticket} still pending after {timeout} s")
            time.sleep(interval)

    def stats(self) -> dict:
        st = mmvm_server_counters()
        _check(load_library().mmvm_server_stats(self.handle, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in mmvm_server_counters._fields_}

    def close(self):
        if self.handle:
            load_library().mmvm_server_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
