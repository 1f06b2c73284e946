"""Compile the FP64 oracle (plain C, OpenMP) in place. Test infrastructure only."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def command():
    # -ffp-contract=off: every FP64 operation rounds as written (no fused multiply-add).
    return ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-fopenmp", "-ffp-contract=off", "-o", LIB, SRC, "-lm"]


def build(force=False):
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    subprocess.run(command(), check=True)
    return LIB
