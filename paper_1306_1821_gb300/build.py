"""Build of the CUDA library libbps.so for sm_103a (nvcc, in-tree, no cmake).

The translation units compile in parallel; the shared library links the
CUDA runtime dynamically so that it shares the process's runtime with PyTorch.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "lib")
LIB = os.path.join(OUT, "libbps.so")
UNITS = ["bps_passes.cu", "bps_draws.cu", "bps_api.cu", "bps_noalloc.cu", "bps_mlp.cu", "bps_yz.cu",
         "bps_mock.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-warn-spills"]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    if verbose and (r.stdout or r.stderr):
        print(r.stdout + r.stderr, flush=True)
    return r


def build(verbose=False, extra=()):
    """Compile csrc/*.cu to lib/libbps.so; returns the library path."""
    os.makedirs(OUT, exist_ok=True)
    objs = []
    cmds = []
    for u in UNITS:
        o = os.path.join(OUT, u.replace(".cu", ".o"))
        objs.append(o)
        cmds.append([nvcc(), *ARCH, *FLAGS, *extra, "-I", os.path.join(HERE, "..", "include"), "-c",
                     os.path.join(SRC, u), "-o", o])
    with ThreadPoolExecutor(len(cmds)) as ex:
        list(ex.map(lambda c: _run(c, verbose), cmds))
    _run([nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", LIB, *objs], verbose)
    return LIB


if __name__ == "__main__":
    build(verbose="-v" in sys.argv)
    print(LIB)
