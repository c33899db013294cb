"""Builds the CUDA library librt_gb300.so in-tree with nvcc for sm_103a.

Each .cu file is compiled on its own (in parallel) and the objects are
linked into one shared library with the CUDA runtime linked statically.
"""
import os
import shutil
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librt_gb300.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["rt_api.cu", "rt_step.cu", "rt_transport.cu", "rt_aux.cu", "rt_adjoint.cu", "rt_noalloc.cu",
           "rt_recon.cu", "rt_groups.cu", "rt_hydro.cu"]
# per-file flags: the gas dynamics round as their plain formulas (no FMA contraction)
FILE_FLAGS = {"rt_hydro.cu": ["--fmad=false"]}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# host code is compiled without FMA contraction so that x86 and Arm hosts
# build bit-identical face geometry
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2,-ffp-contract=off",
         "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]
_lock = threading.Lock()


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librt_gb300.so")
    return exe


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "rt.h"))
    return files


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, extra_flags=()):
    """Compile librt_gb300.so if any source is newer than it; return its path."""
    with _lock:
        deps = _deps()
        if not force and not _stale(LIB, deps):
            return LIB
        os.makedirs(BUILD, exist_ok=True)
        exe = nvcc()

        def compile_one(src):
            obj = os.path.join(BUILD, src.replace(".cu", ".o"))
            cmd = [exe, *ARCH, *FLAGS, *FILE_FLAGS.get(src, []), *extra_flags, "-I", INCLUDE, "-c",
                   os.path.join(CSRC, src), "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
            if verbose and r.stderr:
                print(r.stderr)
            return obj

        with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
            objs = list(ex.map(compile_one, SOURCES))
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [exe, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
