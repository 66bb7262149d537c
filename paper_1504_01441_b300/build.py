"""Build of the in-tree CUDA libraries (sm_103a) with nvcc.

libhdrreg.so exports the C ABI declared in include/hdrreg.h; the Python binding
in this package loads it with ctypes. libhdrreg_probe.so (probe/) is the
benchmark's integer dot-product rate probe, kept out of the registration library.
"""
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libhdrreg.so")
PROBE_SRC = os.path.join(PKG, "probe", "dp4a_rate.cu")
PROBE_LIB = os.path.join(PKG, "probe", "libhdrreg_probe.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared",
         "-Xlinker", "-rpath=/usr/local/cuda/lib64", "--expt-relaxed-constexpr"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale():
    if not os.path.exists(LIB):
        return True
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(out, srcs, extra, verbose):
    tmp = out + ".tmp%d" % os.getpid()
    cmd = [NVCC, *ARCH, *FLAGS, "-I", INCLUDE, "-I", CSRC, *extra, "-o", tmp, *srcs]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, out)


def build(force=False, verbose=False, extra=()):
    if force or not os.path.exists(PROBE_LIB) or \
            os.path.getmtime(PROBE_SRC) > os.path.getmtime(PROBE_LIB):
        _compile(PROBE_LIB, [PROBE_SRC], extra, verbose)
    if force or _stale():
        _compile(LIB, sources(), extra, verbose)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [])
    print(LIB)
