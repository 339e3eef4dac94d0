"""Compile the seeded input generators: a host library (gcc, OpenMP) and a device
library (nvcc, sm_103a). Both are built in-tree under datagen/_build/."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "_build")
HOST_LIB = os.path.join(OUT, "libdatagen_host.so")
DEV_LIB = os.path.join(OUT, "libdatagen_dev.so")

NVCC_ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def host_cmd():
    return ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
            os.path.join(HERE, "datagen_host.c"), "-o", HOST_LIB, "-lm"]


def device_cmd():
    return ["nvcc", *NVCC_ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
            "-shared", "-cudart", "static", os.path.join(HERE, "datagen_device.cu"), "-o", DEV_LIB]


def commands(device=True):
    os.makedirs(OUT, exist_ok=True)
    cmds = [host_cmd()]
    if device:
        cmds.append(device_cmd())
    return cmds


def build(device=True):
    procs = [subprocess.Popen(c) for c in commands(device)]
    for c, p in zip(commands(device), procs):
        if p.wait() != 0:
            raise RuntimeError("datagen build failed: " + " ".join(c))
