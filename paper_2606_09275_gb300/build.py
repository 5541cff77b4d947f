"""Build libmpm_gb300.so in-tree from csrc/*.cu for sm_103a (nvcc, no cmake).

Each translation unit is compiled in parallel with one -gencode; the shared
library lands next to this file, where the binding loads it.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INC = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libmpm_gb300.so")
OBJ = os.path.join(HERE, "_build")
UNITS = ["mpm_ctx", "mpm_cub", "mpm_build", "mpm_assemble", "mpm_solve", "mpm_step", "mpm_adjoint",
         "mpm_mg", "mpm_peak"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# the mesh build decides discrete events (overlaps, splits, marks) from box
# arithmetic: keep it to separately rounded multiplies and adds
PER_UNIT = {"mpm_build": ["--fmad=false"]}


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _deps():
    files = [os.path.join(SRC, f) for f in os.listdir(SRC)]
    files.append(os.path.join(INC, "mpm.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(force=False, verbose=False):
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    cc = nvcc()

    def one(u):
        o = os.path.join(OBJ, u + ".o")
        cmd = [cc] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                             "-I" + INC, "-c", os.path.join(SRC, u + ".cu"), "-o", o]
        cmd += PER_UNIT.get(u, [])
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (u, r.stderr))
        if verbose:
            print(r.stderr)
        return o

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(one, UNITS))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
