"""Compile the synthetic-canvas generator (host C++) in place."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "synth.cpp")
LIB = os.path.join(HERE, "libsynth.so")


def command():
    # -ffp-contract=off: the FP32 blend must round every step the same way on x86 and Arm.
    return ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-ffp-contract=off", "-o", LIB, SRC]


def build(force=False):
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    subprocess.run(command(), check=True)
    return LIB
