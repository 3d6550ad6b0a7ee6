"""The whole path through the C ABI from a C99 program on the GPU (no Python between the caller
and the library): device buffers from cudaMalloc, every schedule, A and b against the oracle's
own C interface (tests/c_abi/gpu_eval_stamp.c)."""
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_runs_every_schedule_against_the_oracle(tmp_path):
    from paper_2604_03079_gb300 import build
    import oracle
    lib = build.build()
    olib = oracle.build()
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    exe = str(tmp_path / "gpu_eval_stamp")
    libdir, odir = os.path.dirname(lib), os.path.dirname(olib)
    cudalib = next(p for p in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib"))
                   if os.path.isdir(p))
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-O2",
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
                    os.path.join(ROOT, "tests", "c_abi", "gpu_eval_stamp.c"), "-o", exe,
                    "-L", libdir, "-l:_libeec.so", "-L", odir, "-l:_liboracle.so",
                    "-L", cudalib, "-lcudart", "-lm",
                    "-Wl,-rpath," + libdir, "-Wl,-rpath," + odir, "-Wl,-rpath," + cudalib],
                   check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", (out.returncode, out.stderr)
