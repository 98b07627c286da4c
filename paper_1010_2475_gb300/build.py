"""Build libmmvm.so in-tree for sm_103a (nvcc, parallel per translation unit).

    python -m paper_1010_2475_gb300.build [--jobs N] [--force]

Every pair-kernel variant (order 0..8, FP64 and FP32) is its own object file
so that they compile in parallel; an object is rebuilt only when a source
file it depends on is newer.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmmvm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
MAX_ORDER_PAIRS = 8


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmmvm.so")


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(INCLUDE, "mmvm.h"))
    return hs


def _n_variants(m: int, p: int) -> int:
    """Mirror of n_variants() in csrc/pair_variants.h."""
    if p == 0:
        return 1
    return 1 if m <= 3 else (2 if m == 7 else (4 if m == 6 else 3))


def _n_slices(m: int, p: int, v: int) -> int:
    """Mirror of variant_spec(m, p, v).nslices in csrc/pair_variants.h."""
    if p == 0:
        return {0: 1, 1: 1, 2: 1, 3: 1, 4: 2, 5: 2, 6: 3, 7: 4, 8: 4}[m]
    if m <= 3:
        return 1
    return {4: [1, 1, 2], 5: [1, 2, 2], 6: [1, 2, 3, 2], 7: [2, 3], 8: [3, 4, 4]}[m][v]


def _units():
    """(source, object, extra flags) for every translation unit."""
    units = []
    for m in range(MAX_ORDER_PAIRS + 1):
        for p in (0, 1):
            for v in range(_n_variants(m, p)):
                for sl in range(_n_slices(m, p, v)):
                    units.append(("pair_inst.cu", f"pair_m{m}_p{p}_v{v}_s{sl}.o",
                                  [f"-DMMVM_INST_M={m}", f"-DMMVM_INST_PREC={p}",
                                   f"-DMMVM_INST_V={v}", f"-DMMVM_INST_S={sl}"]))
    for src in ("pair_registry.cu", "particle_kernels.cu", "order.cu", "api.cu", "calibrate.cu",
                "noalloc.cu", "server.cu", "self_high.cu", "tables.cpp"):
        units.append((src, os.path.splitext(src)[0] + ".o", []))
    return units


def _compile(nvcc, src, obj, extra, force):
    src_path = os.path.join(CSRC, src)
    obj_path = os.path.join(BUILD, obj)
    deps = [src_path] + _headers()
    if (not force and os.path.exists(obj_path)
            and os.path.getmtime(obj_path) >= max(os.path.getmtime(d) for d in deps)):
        return obj_path, "up to date"
    lang = ["-x", "cu"] if src.endswith(".cpp") else []
    cmd = [nvcc, "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC",
           "-I", CSRC, "-I", INCLUDE, *extra, *lang, "-c", src_path, "-o", obj_path]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src} {extra}:\n{res.stdout}\n{res.stderr}")
    return obj_path, "built"


def build(jobs: int | None = None, force: bool = False, verbose: bool = True) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    jobs = jobs or max(1, os.cpu_count() or 1)
    units = _units()
    # heaviest variants first so the pool stays busy
    units.sort(key=lambda u: -int(u[1].split("_m")[1].split("_")[0]) if u[1].startswith("pair_m") else 0)
    stale = [f for f in os.listdir(BUILD) if f.endswith(".o") and f not in {u[1] for u in units}]
    for f in stale:  # objects of variants that no longer exist
        os.remove(os.path.join(BUILD, f))
    objs = []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        futs = [ex.submit(_compile, nvcc, s, o, e, force) for s, o, e in units]
        for f in futs:
            path, status = f.result()
            objs.append(path)
            if verbose and status == "built":
                print(f"[mmvm build] {os.path.basename(path)}", flush=True)
    newest = max(os.path.getmtime(o) for o in objs)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        cmd = [nvcc, *ARCH, "-shared", "-o", LIB, *objs, "-lcudart"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
        if verbose:
            print(f"[mmvm build] linked {LIB}", flush=True)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=None)
    ap.add_argument("--force", action="store_true")
    a = ap.parse_args()
    build(a.jobs, a.force)
    sys.exit(0)
