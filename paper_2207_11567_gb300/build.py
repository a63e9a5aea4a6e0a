"""Build of the CUDA library (sm_103a only): each translation unit is compiled by nvcc in
parallel, then linked into ``libhlbm.so`` next to this file. Object files go to ``_build/``."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhlbm.so")
SOURCES = ["api.cu", "aux_kernels.cu", "stats.cu", "fd_kernels.cu", "fd_tiled.cu", "lb_d2q9.cu", "lb_d3q27_f64.cu",
           "lb_d3q27_f32.cu", "lb_d3q27_f16.cu", "noalloc.cu", "adjoint.cu",
           "flame.cu", "probes.cu", "fd_kernels_vcp.cu", "fd_kernels_mix.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def nvcc():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    path = os.path.join(home, "bin", "nvcc")
    return path if os.path.exists(path) else "nvcc"


def _needs(obj, srcs):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(s) > t for s in srcs)


def build(verbose=False, extra_flags=()):
    """Compile (if stale) and link the library; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(HERE, "..", "include", "hlbm.h"))
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if _needs(o, [s] + headers):
            jobs.append([nvcc(), *FLAGS, *extra_flags, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.returncode

    with ThreadPoolExecutor(max_workers=min(8, max(1, len(jobs)))) as ex:
        codes = list(ex.map(run, jobs))
    if any(codes):
        raise RuntimeError("nvcc failed")
    if jobs or not os.path.exists(LIB) or _needs(LIB, objs):
        tmp = LIB + ".tmp"
        if run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs]) != 0:
            raise RuntimeError("link failed")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
