"""Builds the FP64 CPU oracle (test infrastructure only) with gcc.

The oracle is plain C; this script compiles it into ``oracle/liboracle.so``
next to the source.  Nothing here touches the CUDA library.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "qs_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
           "-D_GNU_SOURCE", SRC, "-o", tmp, "-lm"]
    # OpenMP only splits independent pair updates across threads; without
    # it the oracle is the same program, single-threaded.
    if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:]).returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
