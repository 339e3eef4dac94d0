"""Compile the CUDA library libmsi.so (sm_103a) in-tree:
paper_2009_00786_gb300/_build/libmsi.so. One nvcc process per translation unit,
in parallel, then one link."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libmsi.so")
SOURCES = ["msi_api.cu", "msi_build.cu", "msi_query.cu", "msi_noalloc.cu", "msi_serve.cu", "msi_persist.cu", "msi_merge.cu", "msi_tc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-Xptxas", "-v"]


def compile_commands():
    cmds = []
    for src in SOURCES:
        obj = os.path.join(OUT, src.replace(".cu", ".o"))
        cmds.append((["nvcc", *ARCH, *FLAGS, "-dc" if False else "-c", os.path.join(CSRC, src), "-o", obj], obj))
    return cmds


def build(verbose=False):
    os.makedirs(OUT, exist_ok=True)
    cmds = compile_commands()
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for c, _ in cmds]
    logs = []
    for (c, _), p in zip(cmds, procs):
        out, _ = p.communicate()
        logs.append(out.decode(errors="replace"))
        if p.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(c) + "\n" + logs[-1])
    link = ["nvcc", *ARCH, "-shared", "-cudart", "static", "-o", LIB, *[o for _, o in cmds]]
    subprocess.run(link, check=True)
    if verbose:
        print("\n".join(logs))
    return "\n".join(logs)
