"""In-tree build of the CUDA library (libmrf_gb300.so) for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library with the static CUDA runtime. Output: ``_build/`` beside this
file (``_build_check/`` for the bounds-checked variant; both git-ignored). No
CMake, no torch extension machinery.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
# MRF_BUILD_VARIANT=check selects the bounds-checked build (-DMRF_CHECK: a
# failed device index check sets the context's error flag, reported by
# mrf_stream_sync, and skips the access), kept in its own folder
VARIANT = os.environ.get("MRF_BUILD_VARIANT", "")
if VARIANT not in ("", "check"):
    raise ValueError(f"MRF_BUILD_VARIANT must be empty or 'check', not {VARIANT!r}")
BUILD = os.path.join(HERE, "_build_check" if VARIANT == "check" else "_build")
LIB = os.path.join(BUILD, "libmrf_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
_lock = threading.Lock()


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the MRF library needs the CUDA toolkit to build")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "mrf.h"),
                                                                 os.path.abspath(__file__)]


def is_stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile every CUDA/C++ source for sm_103a and link libmrf_gb300.so."""
    with _lock:
        if not force and not is_stale():
            return LIB
        os.makedirs(BUILD, exist_ok=True)
        nvcc = _nvcc()
        common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo", "--expt-relaxed-constexpr",
                  "-I", os.path.join(HERE, "..", "include")] + list(extra_flags)
        if VARIANT == "check":
            common.append("-DMRF_CHECK")
        if verbose:
            common += ["-Xptxas", "-v"]

        def compile_one(src):
            obj = os.path.join(BUILD, os.path.basename(src) + ".o")
            cmd = [nvcc, *ARCH, *common, "-c", src, "-o", obj]
            if src.endswith(".cpp"):
                cmd = [nvcc, *common, "-x", "c++", "-c", src, "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
            return obj, (r.stdout + r.stderr)

        with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
            results = list(ex.map(compile_one, sources()))
        objs = [o for o, _ in results]
        logs = "".join(l for _, l in results)
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
        if verbose:
            print(logs)
        return LIB


if __name__ == "__main__":
    import sys
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
