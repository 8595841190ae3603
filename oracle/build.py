"""Compile the FP64 oracle (plain C) into oracle/_build/liboracle.so.

The oracle is test infrastructure: the library built here is loaded only by the
tests, the smoke check and the benchmark's CPU-baseline leg.  No FMA contraction
(-ffp-contract=off) so that each floating-point operation in the source is one
IEEE operation on x86-64 and aarch64 alike.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "moldy_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def compile_source(src: str, out: str) -> str:
    """Compile one oracle source file into a shared library at `out` (the flags of the oracle)."""
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    compile_source(SRC, tmp)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
