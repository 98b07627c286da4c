"""The C-ABI library builds, loads and exports every symbol include/mmvm.h declares.

No compute calls (this runs without a GPU).  The header is parsed for its
function declarations so a new entry point cannot be forgotten in the binding.
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mmvm.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mmvm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_1010_2475_gb300 as mm
    from paper_1010_2475_gb300 import build

    build.build(verbose=False)
    return mm.load_library()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert "mmvm_create" in names and "mmvm_step" in names
    for name in names:
        assert hasattr(lib, name), name
    import paper_1010_2475_gb300 as mm

    assert sorted(mm.EXPORTS) == names


def test_exports_have_c_linkage(lib):
    import paper_1010_2475_gb300 as mm

    out = subprocess.run(["nm", "-D", "--defined-only", mm.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    syms = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    for name in _declared():
        assert name in syms, f"{name} not exported unmangled"


def test_pure_host_entry_points(lib):
    import paper_1010_2475_gb300 as mm

    assert lib.mmvm_num_moments(6) == 28
    assert lib.mmvm_num_moments(60) == 1891
    assert lib.mmvm_num_particles(None) == 0
    # an invalid config is rejected before any device call
    cfg = mm.mmvm_config(-1, 0, 1.0, 0.0, 0, 0)
    h = ctypes.c_void_p()
    assert lib.mmvm_create(ctypes.byref(cfg), ctypes.byref(h)) == mm.MMVM_E_INVALID_ARG
    assert b"order" in lib.mmvm_last_error()
    cfg = mm.mmvm_config(2, 7, 1.0, 0.0, 0, 0)
    assert lib.mmvm_create(ctypes.byref(cfg), ctypes.byref(h)) == mm.MMVM_E_INVALID_ARG
    cfg = mm.mmvm_config(99, 0, 1.0, 0.0, 0, 0)
    assert lib.mmvm_create(ctypes.byref(cfg), ctypes.byref(h)) == mm.MMVM_E_UNSUPPORTED
    cfg = mm.mmvm_config(2, 0, -1.0, 0.0, 0, 0)
    assert lib.mmvm_create(ctypes.byref(cfg), ctypes.byref(h)) == mm.MMVM_E_INVALID_ARG


def test_request_footprint_host_only(lib):
    """Admission accounting of the server: FP64 state (step start, stage, RK4
    sum), source records padded to groups of 32, one block of partial sums per
    1024-source chunk, work lists."""
    import paper_1010_2475_gb300 as mm

    def expected(order, prec, n):
        K = (order + 1) * (order + 2) // 2
        NB = (2 * order + 1) * (2 * order + 2) // 2 - 1 if order > 0 else 2
        hdr = 4 if prec == mm.MMVM_MIXED_FP32 else 2
        eb = 4 if prec == mm.MMVM_MIXED_FP32 else 8
        far = 2 * (order + 1) if prec == mm.MMVM_MIXED_FP32 else 0
        align = 16 // eb
        rec = -(-(hdr + K + far) // align) * align
        slots = -(-n // 32) * 32
        chunks = 0 if n <= 1 else min(-(-n // 1024), 16)
        items = (slots // 32 + 1) * max(chunks, 1) * 16 + n * 8 + slots // 32 * 4 + 64
        nt = order + [8, 10, 12, 14, 15, 17, 18, 19, 21][min(order, 8)] + 1  # expansion terms
        gl = -(-(8 + 2 * nt) // 4) * 4  # floats per group record
        order = slots * 28 + slots // 32 * 4 * gl + 32 if prec == mm.MMVM_MIXED_FP32 else 0
        return 6 * n * (2 + K) * 8 + slots * rec * eb + chunks * NB * n * 8 + items + order

    for order, prec, n in [(2, 1, 64), (4, 1, 4096), (8, 1, 8192), (6, 0, 1000), (10, 1, 1),
                           (0, 0, 2)]:
        assert mm.mmvm_request_footprint(order, prec, n) == expected(order, prec, n)
    assert (mm.mmvm_request_footprint(8, 1, 8192) > mm.mmvm_request_footprint(4, 1, 8192)
            > mm.mmvm_request_footprint(4, 1, 4096))
    with pytest.raises(mm.MMVMError):
        mm.mmvm_request_footprint(4, 1, 0)
    with pytest.raises(mm.MMVMError):
        mm.mmvm_request_footprint(4, 5, 10)


def test_missing_library_fails_loudly(tmp_path):
    import paper_1010_2475_gb300 as mm

    with pytest.raises(RuntimeError, match="missing"):
        old = mm._lib_handle
        mm._lib_handle = None
        try:
            mm.load_library(str(tmp_path / "libmmvm.so"))
        finally:
            mm._lib_handle = old
