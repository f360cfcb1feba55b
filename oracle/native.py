"""Builds the plain-C part of the oracle (rows.c) into oracle/_rows.so.

Test infrastructure only (see the package docstring)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rows.c")
LIB = os.path.join(HERE, "_rows.so")


def build():
    if not os.path.exists(SRC):
        return None
    tmp = LIB + ".tmp"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, SRC, "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB
