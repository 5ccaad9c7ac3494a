"""Compile the CUDA library (libhamr.so) for sm_103a, in-tree under _build/.

Each translation unit is compiled in parallel with nvcc; the objects are linked into one
shared library against the shared CUDA runtime.  No cmake, one -gencode.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libhamr.so")
SOURCES = ["api.cu", "kernels_plain.cu", "kernels_fused_sc.cu", "kernels_fused_l10.cu", "kernels_misc.cu", "noalloc.cu",
           "multiscale.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhamr")
    return exe


def flags():
    return [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
            "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, extra=()):
    os.makedirs(OUT, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(ROOT, "include", "hamr.h"))
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT, src.replace(".cu", ".o"))
        if force or extra or _stale(o, [s, *headers]):
            # the fused kernels write every multiply-add out (identical rounding in every
            # instantiation, see kernels_fused.cuh)
            fmad = ["-fmad=false"] if src.startswith("kernels_fused") else []
            # the multiscale driver decides on the host when the window moves; its host
            # arithmetic rounds every multiply and add on its own on every platform
            if src == "multiscale.cu":
                fmad = ["-Xcompiler", "-ffp-contract=off"]
            jobs.append([nvcc(), *flags(), *fmad, *extra, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for msg in ex.map(run, jobs):
            if verbose and msg:
                print(msg, file=sys.stderr)
    objs = [os.path.join(OUT, s.replace(".cu", ".o")) for s in SOURCES]
    if jobs or not os.path.exists(LIB):
        tmp = LIB + ".tmp%d" % os.getpid()
        run([nvcc(), *ARCH, "-shared", "-cudart", "shared", *objs, "-lcufft", "-o", tmp])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=("-Xptxas", "-v") if "--ptxas" in sys.argv else ()))
