"""Build the in-tree C-ABI library libfdetd.so for sm_103a (GB300).

Host C++ (plan builder, eigen-solver) is compiled with g++, CUDA sources with
nvcc -gencode arch=compute_103a,code=sm_103a, all translation units in parallel,
then linked with nvcc -shared against the shared CUDA runtime.  Output:
paper_2605_12132_gb300/lib/libfdetd.so (git-ignored).
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INC = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "lib")
BUILD_DIR = os.path.join(ROOT, "_build")
LIB = os.path.join(OUT_DIR, "libfdetd.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _run(cmd):
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError("command failed:\n" + " ".join(cmd) + "\n" + p.stdout)
    return p.stdout


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def build(verbose=False, extra_nvcc=()):
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()
    cmds, objs = [], []
    for f in sources():
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD_DIR, f + ".o")
        objs.append(obj)
        if f.endswith(".cpp"):
            cmds.append(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-I", INC, "-I", CSRC,
                         "-c", src, "-o", obj])
        else:
            cmds.append([nvcc, ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
                         "-I", INC, "-I", CSRC, *extra_nvcc, "-c", src, "-o", obj])
    with ThreadPoolExecutor(max_workers=min(8, len(cmds))) as ex:
        outs = list(ex.map(_run, cmds))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    _run([nvcc, ARCH, "-shared", "-cudart", "shared", "-o", LIB, *objs])
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, extra_nvcc=["-Xptxas", "-v"] if "-v" in sys.argv else []))
