"""Build the CUDA library in-tree: ``paper_2310_16238_gb300/_build/libcoxgb.so`` (sm_103a).

Each ``csrc/*.cu`` is compiled in parallel with nvcc for ``sm_103a`` only, then linked
into one shared library with a C ABI (declared in ``include/cox.h``). No torch types cross
the ABI; the Python binding (``cox.py``) loads the library with ctypes.

``python -m paper_2310_16238_gb300.build --trace`` builds the diagnostic variant
(``_build/trace/libcoxgb.so``, compiled with -DCOXGB_TRACE: per-step phase stamps of the
resident and incremental kernels, printed when COXGB_PHASE_TRACE=<steps> is set). The binding
loads it instead of the default library when COXGB_LIBRARY names its path.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libcoxgb.so")
TRACE_LIB = os.path.join(BUILD, "trace", "libcoxgb.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcoxgb")
    return exe


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
                   "-I", CSRC, *extra]


def _stale(lib: str, sources) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = list(sources) + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "cox.h"), __file__]
    return any(os.path.getmtime(s) > t for s in deps)


def build(force: bool = False, verbose: bool = False, extra=(), trace: bool = False) -> str:
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    lib = TRACE_LIB if trace else LIB
    if trace:
        extra = [*extra, "-DCOXGB_TRACE"]
    if not force and not _stale(lib, sources):
        return lib
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    exe = nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + f".{os.getpid()}.o")
        cmd = [exe, *_flags(extra), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(sources))) as ex:
        objs = list(ex.map(compile_one, sources))
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([exe, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    for o in objs:
        os.remove(o)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, trace="--trace" in sys.argv))
