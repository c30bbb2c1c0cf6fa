"""Compile the EMPC oracle (plain C, FP64) into a shared library.

Test infrastructure: builds the checker, never the product path.  The flags
matter for bit-exact parity of the FP32 genome operations: -ffp-contract=off
keeps every a*b+c in the source a separate multiply and add, so the only
fused operations are the explicit fmaf() calls.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "empc_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liborc.so")


def _compile(openmp: bool) -> None:
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", SRC, "-o", LIB + ".tmp", "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True, capture_output=True)
    os.replace(LIB + ".tmp", LIB)


def build(force: bool = False) -> str:
    """Build liborc.so if missing or older than its source; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    try:
        _compile(openmp=True)
    except subprocess.CalledProcessError:
        _compile(openmp=False)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
