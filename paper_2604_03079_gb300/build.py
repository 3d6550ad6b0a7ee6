"""Build the CUDA library ``_libeec.so`` in-tree for sm_103a (GB300).

Every translation unit compiles in parallel with one ``-gencode`` so that a fresh box builds in
well under a minute. ``python -m paper_2604_03079_gb300.build [-v]`` runs it by hand; ``-v``
adds ``-Xptxas -v`` (registers, spills, shared memory per kernel).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "_libeec.so")
SOURCES = ["eec_capi.cpp", "eec_kernels.cu", "eec_gather.cu", "eec_bwd.cu", "eec_color.cu",
           "eec_newton.cu", "eec_lu.cu"]
LIBS = ["-lcusolver", "-lcusparse"]   # the sparse solve of eec_newton_dc
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = [os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]
    for c in cand:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "eec.h"))
    return any(os.path.getmtime(p) > t for p in deps if os.path.exists(p))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    cc = nvcc()
    odir = os.path.join(HERE, "_build")
    os.makedirs(odir, exist_ok=True)
    common = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden", "-cudart", "shared",
                     "-I", os.path.join(HERE, "..", "include")]
    if verbose:
        common += ["-Xptxas", "-v"]
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(odir, src.rsplit(".", 1)[0] + ".o")
        objs.append(obj)
        cmd = [cc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append(f"--- {src}\n{text}")
        elif verbose and text.strip():
            sys.stdout.write(f"--- {src}\n{text}")
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.run([cc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + LIBS,
                   check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
