"""Build the sm_103a library libtqs.so in-tree (nvcc + g++, no cmake).

    python -m paper_2305_14398_gb300.build [--force] [--checked]

Every translation unit compiles in parallel; the shared library lands next to
this file and the objects under _build/.  Rebuilds only what changed.
--checked builds the bounds-checked variant (-DTQS_CHECKED) as
libtqs_checked.so, objects under _build_checked/.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtqs.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libtqs_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    for cand in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    return cu, cpp


def _headers_mtime() -> float:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return max((os.path.getmtime(h) for h in hs), default=0.0)


def _stale(src: str, obj: str, hdr_mtime: float) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return t < os.path.getmtime(src) or t < hdr_mtime


def build(force: bool = False, verbose: bool = False, extra_nvcc=None, checked: bool = False) -> str:
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    build_dir = BUILD_CHECKED if checked else BUILD
    lib_path = LIB_CHECKED if checked else LIB
    if checked:
        extra_nvcc = list(extra_nvcc or []) + ["-DTQS_CHECKED"]
    os.makedirs(build_dir, exist_ok=True)
    cu, cpp = _sources()
    hdr = _headers_mtime()
    jobs = []
    for f in cu:
        src, obj = os.path.join(CSRC, f), os.path.join(build_dir, f + ".o")
        if force or _stale(src, obj, hdr):
            cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "--expt-relaxed-constexpr", "-I", CSRC, "-I", INCLUDE, "-c", src, "-o", obj]
            if extra_nvcc:
                cmd[1:1] = list(extra_nvcc)
            jobs.append(cmd)
    for f in cpp:
        src, obj = os.path.join(CSRC, f), os.path.join(build_dir, f + ".o")
        if force or _stale(src, obj, hdr):
            # -fcx-fortran-rules: complex products without the C99 NaN
            # re-check (finite values give the same results; the host compile
            # multiplies many 2x2 complex matrices)
            jobs.append(["g++", "-O3", "-fcx-fortran-rules", "-std=c++17", "-fPIC", "-pthread", "-Wall",
                         "-I", os.path.join(cuda, "include"),
                         "-I", CSRC, "-I", INCLUDE, "-c", src, "-o", obj])
    objs = [os.path.join(build_dir, f + ".o") for f in cu + cpp]

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stderr

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for msg in ex.map(run, jobs):
                if verbose and msg.strip():
                    print(msg, flush=True)
    if jobs or not os.path.exists(lib_path):
        tmp = lib_path + ".tmp"
        run([nvcc, *ARCH, "-shared", "-Xcompiler", "-pthread", "-o", tmp, *objs, "-lcudart", "-lcuda"])
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
