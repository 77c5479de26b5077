"""Build the CUDA library in-tree: paper_1602_05700_gb300/_build/libhypergrav.so (sm_103a only), and on request its
checked variant _build/libhypergrav_debug.so (compiled with -DHG_DEBUG; loaded instead when HG_DEBUG=1 is set).

Each translation unit of csrc/ is compiled by nvcc in parallel, then linked into one shared library with the CUDA
runtime linked statically, so nothing but the driver is needed at load time.  Rebuilds only what is out of date.
"""
from __future__ import annotations

import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libhypergrav.so")
LIB_DEBUG = os.path.join(BUILD, "libhypergrav_debug.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# host code: no floating-point contraction (the Robin and multipole set-up must round the same on x86 and Arm)
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "-Xcompiler", "-ffp-contract=off",
         "--expt-relaxed-constexpr"]
# per-file device flags: the hydrodynamics is compiled without multiply-add contraction, so that its FP64 instance
# rounds every operation as written (the operation order its ABI header fixes)
FILE_FLAGS = {"hydro.cu": ["-fmad=false"]}


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _newest(paths) -> float:
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, debug: bool = False, both: bool = False) -> str:
    """Compile what is out of date and link.  debug=True builds the checked variant (-DHG_DEBUG, index checks before
    the sub-step kernels' stores) as _build/libhypergrav_debug.so; both=True builds the two variants in one pool.
    Returns the path of the (last) library built."""
    variants = (False, True) if both else (bool(debug),)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")))
    hdr_time = _newest(headers) if headers else 0.0
    nvcc = _nvcc()
    for dbg in variants:
        os.makedirs(os.path.join(BUILD, "obj_debug" if dbg else "obj"), exist_ok=True)

    def obj_of(src, dbg):
        return os.path.join(BUILD, "obj_debug" if dbg else "obj", os.path.basename(src)[:-3] + ".o")

    def compile_one(job):
        src, dbg = job
        obj = obj_of(src, dbg)
        if not force and os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr_time):
            return obj
        tmp = f"{obj}.tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, *FLAGS, *(["-DHG_DEBUG"] if dbg else []), *FILE_FLAGS.get(os.path.basename(src), []),
               "-I", INCLUDE, "-c", src, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}{' (debug)' if dbg else ''}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        os.replace(tmp, obj)
        return obj

    jobs = [(src, dbg) for dbg in variants for src in srcs]
    with ThreadPoolExecutor(max_workers=max(1, min(os.cpu_count() or 8, 16, len(jobs)))) as ex:
        objs = list(ex.map(compile_one, jobs))
    out = LIB
    for dbg in variants:
        lib = LIB_DEBUG if dbg else LIB
        mine = [o for o, (_, d) in zip(objs, jobs) if d == dbg]
        if force or not os.path.exists(lib) or os.path.getmtime(lib) < _newest(mine):
            tmp = lib + f".tmp{os.getpid()}"
            cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *mine]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link failed:\n{r.stderr}")
            os.replace(tmp, lib)
        out = lib
    return out


if __name__ == "__main__":
    print(build(verbose=True))
