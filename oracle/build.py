"""Build step for the oracle's C part (plain gcc, OpenMP, FP64).

TEST INFRASTRUCTURE ONLY: the oracle is loaded by the tests, the smoke check
and the CPU-baseline leg of the benchmark, never by the product path.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "siddon.c")
LIB = os.path.join(HERE, "_siddon.so")


def build(force: bool = False) -> str:
    """Compile siddon.c into oracle/_siddon.so (skipped when up to date)."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
           "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
