"""Build the in-tree CUDA library ``_build/libcgks.so`` for sm_103a.

Translation units (one per kernel configuration plus the host code and the
table generator) compile in parallel with nvcc / g++, then link into one
shared library.  ``python -m paper_2508_13705_gb300.build`` rebuilds.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libcgks.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcgks.so")


def sources():
    cu = sorted(f for f in os.listdir(SRC) if f.endswith(".cu"))
    return [os.path.join(SRC, f) for f in cu], [os.path.join(SRC, "tables.cpp")]


def _stale(lib, deps):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    cu, cpp = sources()
    hdrs = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".cuh", ".h"))]
    hdrs.append(os.path.join(os.path.dirname(HERE), "include", "cgks.h"))
    if not force and not _stale(LIB, cu + cpp + hdrs):
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    objs = []
    cmds = []
    for s in cu:
        o = os.path.join(OUT, os.path.basename(s) + ".o")
        objs.append(o)
        cmds.append([nvcc] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                                     "-c", s, "-o", o])
    for s in cpp:
        o = os.path.join(OUT, os.path.basename(s) + ".o")
        objs.append(o)
        cmds.append(["g++", "-O2", "-fPIC", "-std=c++17", "-c", s, "-o", o])

    def run(c):
        r = subprocess.run(c, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(c), r.stdout, r.stderr))
        if verbose:
            sys.stderr.write(r.stderr)
        return r

    with ThreadPoolExecutor(max_workers=min(len(cmds), os.cpu_count() or 4)) as ex:
        list(ex.map(run, cmds))
    tmp = LIB + ".tmp%d" % os.getpid()
    run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
