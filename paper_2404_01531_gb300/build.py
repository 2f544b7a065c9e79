"""Build libffe.so in-tree with nvcc for sm_103a (GB300).

Each CUDA translation unit is compiled in parallel, then linked into a shared
library next to this file.  Usage: python -m paper_2404_01531_gb300.build
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libffe.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["host.cu", "host_geom.cu", "kernels_dg.cu", "kernels_fd.cu", "kernels_curved.cu", "kernels_adjoint.cu", "kernels_adjoint_fd.cu",
           "kernels_fd_interp.cu", "noalloc.cu"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
         "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def build(verbose=False):
    os.makedirs(BUILD, exist_ok=True)
    procs, objs = [], []
    for s in SOURCES:
        obj = os.path.join(BUILD, s.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [NVCC, *FLAGS, "-c", os.path.join(CSRC, s), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((s, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for s, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((s, out.decode()))
        elif verbose and out:
            print(out.decode())
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(f"--- {s}\n{o}" for s, o in failed))
    cudalib = os.path.join(os.path.dirname(os.path.dirname(NVCC)), "lib64")
    link = [NVCC, "-shared", "-cudart", "shared", "-gencode", "arch=compute_103a,code=sm_103a",
            *objs, "-o", OUT, "-Xlinker", f"-rpath,{cudalib}"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode())
    return OUT


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
