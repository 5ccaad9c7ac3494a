"""Compile the FP64 CPU oracle (test infrastructure only) into oracle/_build/liboracle.so.

Plain gcc, no vendor code: -O2 with OpenMP over sites and -ffp-contract=off so that
every multiply and add rounds on its own, as the formulas are written.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hamr_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(src=SRC, lib=LIB, force=False, extra_flags=()):
    """Compile `src` into the shared library `lib` unless it is newer than the source."""
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    if (not force and not extra_flags and os.path.exists(lib)
            and os.path.getmtime(lib) >= os.path.getmtime(src)):
        return lib
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           *extra_flags, src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
