"""Compile the FP64 CPU oracle (test infrastructure only) into oracle/_build/liboracle.so.

Plain gcc, no vendor code: -O2 with OpenMP over sites and -ffp-contract=off so that
every multiply and add rounds on its own, as the formulas are written.  Two sources: the
atomistic sLLG Heun step (hamr_oracle.c) and the multiscale window (hamr_ms_oracle.c),
sharing the declarations of hamr_oracle.h.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hamr_oracle.c")
MS_SRC = os.path.join(HERE, "hamr_ms_oracle.c")
HDR = os.path.join(HERE, "hamr_oracle.h")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(src=SRC, lib=LIB, force=False, extra_flags=(), ms_src=MS_SRC):
    """Compile `src` and `ms_src` into the shared library `lib` unless it is newer than
    both sources and the shared header."""
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    deps = [src, ms_src, HDR]
    if (not force and not extra_flags and os.path.exists(lib)
            and all(os.path.getmtime(lib) >= os.path.getmtime(d) for d in deps)):
        return lib
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-I" + HERE,
           *extra_flags, src, ms_src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
