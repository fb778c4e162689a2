"""Build the FP64 CPU oracle library (test infrastructure).

Compiles ``oracle/*.c`` with plain gcc into ``oracle/liboracle_glasma.so``.
Floating-point contraction is disabled so that the oracle gives the same
results on x86-64 and aarch64 hosts.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle_glasma.so")
SOURCES = ["su3.c", "rng.c", "field.c", "particles.c", "init.c"]


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, "oracle.h"), os.path.join(HERE, "oracle_internal.h")]
    if not force and os.path.exists(LIB):
        mtime = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= mtime for d in deps):
            return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-Wall", "-Wno-unused-function", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
