"""In-tree build of the CUDA library ``libwombat_gb300.so`` for sm_103a.

nvcc compiles each translation unit (one -gencode, in parallel) and links
a shared library next to this file under ``_build/``.  No cmake."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libwombat_gb300.so")
SOURCES = ["wb_sweep.cu", "wb_stages.cu", "wb_capi.cu", "wb_batch.cu"]
HEADERS = ["wb_device.cuh", "wb_internal.h", "wb_units.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libwombat_gb300")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Build the library; checked=True builds the index-checked variant
    (-DWB_CHECKED) under _build/checked/."""
    out = os.path.join(OUT, "checked") if checked else OUT
    lib_path = os.path.join(out, "libwombat_gb300.so")
    flags = FLAGS + (["-DWB_CHECKED"] if checked else [])
    os.makedirs(out, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + \
        [os.path.join(os.path.dirname(HERE), "include", "wombat.h")]
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(out, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            jobs.append([nvcc(), *ARCH, *flags, "-c", s, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            futs = [ex.submit(subprocess.run, j, capture_output=True, text=True) for j in jobs]
            for j, f in zip(jobs, futs):
                r = f.result()
                if r.returncode != 0:
                    raise RuntimeError("nvcc failed: " + " ".join(j) + "\n" + r.stderr[-4000:])
                if verbose and r.stderr:
                    print(r.stderr)
    if force or jobs or _stale(lib_path, objs):
        tmp = lib_path + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed: " + r.stderr[-4000:])
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force=True, verbose=True))
