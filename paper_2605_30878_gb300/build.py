"""Compile the CUDA library (csrc/*.cu) for sm_103a into _build/liblbm.so, and
the same sources with LBM_DEBUG_BOUNDS into _build/liblbm_debug.so (every
index the kernels compute is range-checked; a bad one sets an error bit and
the access is skipped).

The translation units compile in parallel with nvcc and link into one shared
library each, with the CUDA runtime linked statically; the Python binding
loads one of them with ctypes.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblbm.so")
LIB_DEBUG = os.path.join(OUT_DIR, "liblbm_debug.so")
SOURCES = ["lbm_api.cu", "lbm_kern_f32.cu", "lbm_kern_f64.cu", "lbm_kern_f16.cu", "lbm_noalloc.cu", "lbm_debug.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# FP64 kernels round every multiply and add separately, as the FP64 oracle does.
EXTRA = {"lbm_kern_f64.cu": ["-fmad=false"]}
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "-I" + CSRC, "-I" + os.path.join(ROOT, "include")]
VARIANTS = {LIB: ("release", []), LIB_DEBUG: ("debug", ["-DLBM_DEBUG_BOUNDS"])}


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "lbm.h")]


def _stale(lib):
    return not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(p) for p in _deps())


def build(force: bool = False, verbose: bool = False, debug: bool = True) -> str:
    """Build liblbm.so (and, with debug=True, liblbm_debug.so) if missing or
    older than any source; return the path of liblbm.so."""
    os.makedirs(OUT_DIR, exist_ok=True)
    libs = [LIB, LIB_DEBUG] if debug else [LIB]
    todo = [lib for lib in libs if force or _stale(lib)]
    if not todo:
        return LIB
    nvcc = _nvcc()

    def compile_one(job):
        lib, src = job
        tag, defs = VARIANTS[lib]
        os.makedirs(os.path.join(OUT_DIR, tag), exist_ok=True)
        obj = os.path.join(OUT_DIR, tag, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *defs, *EXTRA.get(src, []), "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s (%s):\n%s%s" % (src, tag, r.stdout, r.stderr))
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    jobs = [(lib, src) for lib in todo for src in SOURCES]
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        objs = list(ex.map(compile_one, jobs))
    for lib in todo:
        mine = [o for (l_, _), o in zip(jobs, objs) if l_ == lib]
        tmp = lib + ".tmp%d" % os.getpid()
        r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *mine, "-cudart", "static"], capture_output=True,
                           text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
