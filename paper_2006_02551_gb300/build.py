"""Build the in-tree shared library ``_lib/libwadg.so`` for sm_103a.

Host set-up (C++) is compiled with g++, the kernels and the C ABI with nvcc
(-gencode arch=compute_103a,code=sm_103a), in parallel, then linked against
the CUDA runtime.  No cmake; a build takes well under a minute.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libwadg.so")
# diagnostic build with device-side index checks (-DWADG_CHECKED)
LIB_CHECKED = os.path.join(OUT_DIR, "libwadg_checked.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nv = shutil.which("nvcc")
    if nv:
        return os.path.dirname(os.path.dirname(nv))
    raise RuntimeError("nvcc not found")


def _sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    return cu, cpp


def _stale(lib):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    for d in (CSRC, os.path.join(os.path.dirname(HERE), "include")):
        for f in os.listdir(d):
            if os.path.getmtime(os.path.join(d, f)) > t:
                return True
    return False


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile and link the library; checked=True builds the diagnostic
    variant with device-side index checks (a separate file and object dir)."""
    lib = LIB_CHECKED if checked else LIB
    build_dir = BUILD_DIR + ("_checked" if checked else "")
    extra = ["-DWADG_CHECKED"] if checked else []
    if not force and not _stale(lib):
        return lib
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(build_dir, exist_ok=True)
    cu, cpp = _sources()
    inc = ["-I", CSRC, "-I", os.path.join(os.path.dirname(HERE), "include")]
    jobs = []
    for f in cu:
        o = os.path.join(build_dir, f + ".o")
        jobs.append([nvcc, ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", *extra,
                     "-Xptxas", "-v" if verbose else "-O3", *inc, "-c",
                     os.path.join(CSRC, f), "-o", o])
    for f in cpp:
        o = os.path.join(build_dir, f + ".o")
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", *inc, "-c",
                     os.path.join(CSRC, f), "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        results = list(ex.map(run, jobs))
    for cmd, r in results:
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        if r.returncode != 0:
            raise RuntimeError("compile failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    objs = [cmd[cmd.index("-o") + 1] for cmd, _ in results]
    tmp = lib + ".tmp"
    link = [nvcc, ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: " + r.stdout + r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
