"""Build the FP64 CPU oracle (test infrastructure) into oracle/liboracle.so.

Compiled with -ffp-contract=off so that x86-64 and aarch64 hosts round the
same expressions the same way (no fused multiply-add contraction), and with
-fno-strict-aliasing: gcc 13 at -O2 on aarch64 mis-assembled the moment
matrix of the polynomial helpers under type-based alias analysis (the same
source was correct at -O1, with -fno-strict-aliasing, and on x86-64).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gks_oracle.c")
OUT = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "gks_oracle.h"))
    ):
        return OUT
    tmp = OUT + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-strict-aliasing", "-fno-fast-math", "-fPIC", "-shared",
           "-D_DEFAULT_SOURCE", "-Wall", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
