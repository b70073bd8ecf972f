"""Compile the C-ABI shared library libbura.so in-tree with nvcc for sm_103a.

Sources live in csrc/; the translation units are compiled in parallel and linked with
``nvcc -shared``.  The library is rebuilt when a source or header is newer than it.  Extra nvcc flags
(for instance a -D of a tuning macro) can be given in the environment variable BURA_NVCC_FLAGS.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libbura.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["rational.cpp", "kernels_f32.cu", "kernels_f64.cu", "kernels_tma.cu", "kernels_df.cu", "outer.cu", "fdiag.cu", "strips.cu", "sweep3d.cu",
           "solver.cu", "noalloc.cu", "serve.cpp"]
HEADERS = ["kernels.cuh", "kernels_impl.cuh", "tma.cuh", "guard.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "bura.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src):
    out = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [_nvcc(), "-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
           "-I" + os.path.join(ROOT, "include"), *ARCH, *os.environ.get("BURA_NVCC_FLAGS", "").split(), "-c",
           os.path.join(CSRC, src), "-o", out]
    if src.endswith(".cpp"):
        cmd.insert(1, "-x")
        cmd.insert(2, "c++")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    return out


def build(force=False, verbose=True):
    """Build libbura.so if needed; returns its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [_nvcc(), "-shared", *ARCH, "-o", tmp, *objs, "-lcudart_static", "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB, file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv)
