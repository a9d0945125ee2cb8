"""The boundary from plain C: tests/c/abi_laplacian.c includes only include/spmv_gb300.h and
the CUDA runtime header, links the built library, and drives create / tune / run /
run_host / destroy with raw pointers (no Python or PyTorch in the caller). Compiling and
linking needs no GPU; running it does."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "abi_laplacian.c")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _compile(out_dir) -> str:
    from paper_1711_05487_gb300 import buildlib
    lib_dir = os.path.dirname(buildlib.build())
    cudart_dir = os.path.join(CUDA, "lib64")
    exe = os.path.join(str(out_dir), "abi_laplacian")
    cmd = ["gcc", "-std=c11", "-O2", "-Wall", "-Werror", "-o", exe, SRC,
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           "-L", lib_dir, "-lspmv_gb300", "-L", cudart_dir, "-lcudart",
           f"-Wl,-rpath,{lib_dir}", f"-Wl,-rpath,{cudart_dir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


@pytest.mark.skipif(shutil.which("gcc") is None or
                    not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime_api.h")),
                    reason="needs gcc and the CUDA runtime headers")
def test_c_program_compiles_and_links(tmp_path):
    assert os.path.exists(_compile(tmp_path))


@pytest.mark.gpu
def test_c_program_drives_the_library(tmp_path):
    exe = _compile(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok"), r.stdout
