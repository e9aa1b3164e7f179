"""Build libmhd.so in-tree with nvcc for sm_103a (no JIT, no torch extension)."""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))
HDR = sorted(glob.glob(os.path.join(HERE, "csrc", "*.cuh"))) + [os.path.join(HERE, "..", "include", "mhd.h")]
LIB = os.path.join(HERE, "libmhd.so")
DEBUG_LIB = os.path.join(HERE, "libmhd_debug.so")  # MHD_BOUNDS_CHECK: every checked index recorded (mhd_debug_oob)
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "--expt-relaxed-constexpr"]


def stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in SRC + HDR)


def _build_one(lib: str, defines, objdir: str, verbose: bool) -> None:
    os.makedirs(objdir, exist_ok=True)
    objs = []
    procs = []
    for src in SRC:
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmd = [NVCC, *FLAGS, *defines, "-c", src, "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for src, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0 or verbose:
            sys.stderr.write(out.decode())
        if pr.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}")
    tmp = lib + ".tmp"
    subprocess.check_call([NVCC, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", *objs, "-o", tmp,
                           "-lcudart"])
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False, debug: bool = True) -> str:
    """Build libmhd.so and (debug=True) its index-checking twin libmhd_debug.so."""
    if force or stale(LIB):
        _build_one(LIB, [], os.path.join(HERE, "_build"), verbose)
    if debug and (force or stale(DEBUG_LIB)):
        _build_one(DEBUG_LIB, ["-DMHD_BOUNDS_CHECK"], os.path.join(HERE, "_build_debug"), verbose)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
