"""Compile the FP64 CPU oracle (plain C) into oracle/_build/liborc.so.

Test infrastructure: the oracle is the independent checker of the GPU path.
Building it is not using it; only tests/, ``__graft_entry__.smoke()`` and the
cpu_baseline / reference legs of bench.py load the library.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["orc_kernels.c", "orc_quad.c", "orc_assemble.c", "orc_solve.c", "orc_potentials.c"]
LIB = os.path.join(HERE, "_build", "liborc.so")


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, "orc.h")]
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in deps)):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
