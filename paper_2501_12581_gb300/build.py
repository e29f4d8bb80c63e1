"""Builds the in-tree CUDA library libmboit.so for sm_103a with nvcc.

Seven translation units compiled in parallel, linked with a static CUDA
runtime; output in ``paper_2501_12581_gb300/_lib/``.  nvcc cross-compiles, so
this runs on a machine without a GPU.
"""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libmboit.so")
UNITS = ["mboit_api.cu", "mboit_kernels.cu", "mboit_grid.cu", "mboit_grid_frame.cu", "mboit_grid_power.cu", "mboit_units.cu",
         "mboit_units_trig.cu", "mboit_units_power.cu", "mboit_units_frame.cu", "mboit_grid_multi.cu", "mboit_multi_amr.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-I", INC, "-I", SRC]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libmboit")
    return exe


def _sources():
    srcs = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".cu", ".cuh", ".h"))]
    return srcs + [os.path.join(INC, "mboit.h"), __file__]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force=False, verbose=False, extra=()):
    """Compiles libmboit.so if a source is newer than it; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    exe = nvcc()
    objs, procs = [], []
    for u in UNITS:
        obj = os.path.join(OUT_DIR, u.replace(".cu", f".{os.getpid()}.o"))
        cmd = [exe, *ARCH, *FLAGS, *extra, "-c", os.path.join(SRC, u), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), u))
        objs.append(obj)
    errs = []
    for p, u in procs:
        out = p.communicate()[0].decode(errors="replace")
        if p.returncode != 0:
            errs.append(f"{u}:\n{out}")
        elif verbose and out.strip():
            print(out, file=sys.stderr)
    if errs:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errs))
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call([exe, *ARCH, "-shared", "-o", tmp, *objs])
    for o in objs:
        os.remove(o)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
