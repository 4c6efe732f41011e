"""Build the in-tree CUDA library ``libcosm.so`` for sm_103a.

Each translation unit is compiled in parallel with nvcc (one -gencode,
arch=compute_103a,code=sm_103a, -lineinfo); the objects are linked into a
shared library with the CUDA runtime linked statically. Nothing is
installed; the library sits next to this file.

``build(checked=True)`` also links ``libcosm_checked.so``: the same library
with the kernels compiled with COSM_CHECKS, whose device code validates the
indices it is given (a stand-in for a memory checker; see cosm_kernels.cu).
The package loads it instead of libcosm.so when the environment variable
COSM_LIBRARY is "checked".
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libcosm.so")
LIB_CHECKED = os.path.join(HERE, "libcosm_checked.so")
BUILD = os.path.join(HERE, "_build")
GENCODE = "arch=compute_103a,code=sm_103a"
SOURCES = ["cosm_kernels.cu", "cosm_runtime.cu", "cosm_server.cu", "cosm_static.cu", "cosm_graph.cpp"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcosm.so")
    return cand


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "cosm.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-lineinfo"]
    procs = []
    objs = []
    for src in SOURCES:
        # the checked library differs in the kernels only
        tag = ".checked" if checked and src == "cosm_kernels.cu" else ""
        obj = os.path.join(BUILD, src + tag + ".o")
        objs.append(obj)
        if not force and checked and not tag and os.path.exists(obj) and not _stale(obj):
            continue  # shared with libcosm.so and up to date
        cmd = [nv, "-c", os.path.join(CSRC, src), "-o", obj] + common
        if tag:
            cmd += ["-DCOSM_CHECKS"]
        if src.endswith(".cu"):
            cmd += ["-gencode", GENCODE]
            if verbose:
                cmd += ["-Xptxas", "-v"]
        else:
            cmd += ["-x", "c++"]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call([nv, "-shared", "-o", tmp] + objs + ["-gencode", GENCODE, "-cudart", "static"])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
