"""Builds libqfdtd.so in-tree with nvcc for sm_103a (no cmake, no torch extension).

The translation units are compiled in parallel and linked into
``paper_2211_10185_gb300/lib/libqfdtd.so``.  Run ``python -m paper_2211_10185_gb300.build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
OBJDIR = os.path.join(LIBDIR, "obj")
LIBNAME = "libqfdtd.so"
SOURCES = ["qf_fft_f32.cu", "qf_fft_group.cu", "qf_fft_group_t1.cu", "qf_fft_group_p1.cu", "qf_fft_f64.cu", "qf_fft2.cu", "qf_fft2_n128.cu", "qf_stencil.cu", "qf_fields.cu", "qf_api.cu", "qf_static.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC,-O2",
         "-Xptxas", "-v"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def library_path() -> str:
    return os.path.join(LIBDIR, LIBNAME)


def _compile(src: str, verbose: bool) -> str:
    obj = os.path.join(OBJDIR, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    log = os.path.join(OBJDIR, os.path.splitext(src)[0] + ".log")
    with open(log, "w") as f:
        f.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{res.stderr[-4000:]}")
    if verbose:
        print(f"compiled {src}", flush=True)
    return obj


def build(verbose: bool = False, force: bool = False) -> str:
    """Compiles and links the library if any source is newer than it; returns its path."""
    os.makedirs(OBJDIR, exist_ok=True)
    lib = library_path()
    deps = [os.path.join(CSRC, s) for s in os.listdir(CSRC)]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "qfdtd.h"))
    if not force and os.path.exists(lib):
        newest = max(os.path.getmtime(d) for d in deps)
        if os.path.getmtime(lib) >= newest:
            return lib
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr[-4000:]}")
    os.replace(tmp, lib)
    if verbose:
        print(f"linked {lib}", flush=True)
    return lib


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv)
