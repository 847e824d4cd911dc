"""In-tree build of the CUDA library ``lib/libddi_gb300.so`` for sm_103a.

Host tables (``csrc/tables.cpp``) are compiled by the host compiler with
-ffp-contract=off (their bit-exact reproducibility depends on it); the CUDA
translation units by nvcc for ``compute_103a/sm_103a`` only.  Units compile in
parallel; the library is rebuilt when any source is newer than it.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libddi_gb300.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

CU_SOURCES = ["fft.cu", "fft_nufft.cu", "nufft.cu", "plan.cu", "gpe.cu", "batch.cu", "noalloc.cu"]
CPP_SOURCES = ["tables.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _sources():
    srcs = [os.path.join(CSRC, f) for f in CU_SOURCES + CPP_SOURCES]
    srcs += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    srcs.append(os.path.join(INCLUDE, "ddi.h"))
    return srcs


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def _run(cmd):
    proc = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if proc.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + proc.stdout)
    return proc.stdout


def build(force=False, verbose=False):
    """Compile every unit and link the shared library; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    nvcc = _nvcc()
    objs = []
    cmds = []
    for f in CU_SOURCES:
        obj = os.path.join(LIBDIR, f + ".o")
        objs.append(obj)
        cmds.append([nvcc] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                                     "-I" + INCLUDE, "-c", os.path.join(CSRC, f), "-o", obj])
    for f in CPP_SOURCES:
        obj = os.path.join(LIBDIR, f + ".o")
        objs.append(obj)
        cxx = shutil.which("g++") or "g++"
        cmds.append([cxx, "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math", "-I" + INCLUDE,
                     "-c", os.path.join(CSRC, f), "-o", obj])
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        outs = list(ex.map(_run, cmds))
    if verbose:
        for o in outs:
            sys.stdout.write(o)
    tmp = LIB + ".tmp"
    _run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
