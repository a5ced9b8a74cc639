"""The C ABI from plain C99: the example program compiles and links against
libsbbf.so and the CUDA runtime (any machine), and on a GB300 it runs and
checks its own results (members found, false-positive rate, union, device
key hashing, serialization round trip)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2101_01719_gb300")
SRC = os.path.join(PKG, "examples", "sbbf_example.c")


def _cuda_home():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _build(tmp):
    from paper_2101_01719_gb300 import build
    build.build()
    cuda = _cuda_home()
    exe = os.path.join(tmp, "sbbf_example")
    cmd = ["gcc", "-std=c99", "-O2", "-Wall", "-Wextra", "-Werror",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"), SRC,
           "-L", PKG, "-lsbbf", "-L", os.path.join(cuda, "lib64"), "-lcudart",
           "-Wl,-rpath," + PKG, "-Wl,-rpath," + os.path.join(cuda, "lib64"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_example_compiles_and_links(tmp_path):
    assert os.path.exists(_build(str(tmp_path)))


@pytest.mark.gpu
def test_example_runs(tmp_path):
    exe = _build(str(tmp_path))
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "members 1000000/1000000" in r.stdout
    assert "union-ok 1 keys-ok 1 serialize-ok 1" in r.stdout
