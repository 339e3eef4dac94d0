"""Compile the CPU oracle (plain C, OpenMP) in-tree: oracle/_build/liboracle.so.
Test infrastructure: only tests, the smoke check and the benchmark's CPU-baseline
leg load it."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "liboracle.so")


def command():
    return ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
            "-shared", os.path.join(HERE, "oracle.c"), "-o", LIB, "-lm"]


def build():
    os.makedirs(OUT, exist_ok=True)
    subprocess.run(command(), check=True)
