"""The C ABI from plain C: include/dinr_example.c compiles as C11 with
every warning an error against include/dinr.h and links against the
in-tree libdinr.so (CPU); on a GPU it trains a small network on the exact
projections of a sphere and its loss falls below a tenth of the first
step's (exit status 0)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "include", "dinr_example.c")
LIBDIR = os.path.join(ROOT, "paper_2404_19075_b300")


def _build(tmp_path):
    if not shutil.which("gcc"):
        pytest.skip("needs gcc")
    if not os.path.exists(os.path.join(LIBDIR, "libdinr.so")):
        pytest.skip("libdinr.so is not built")
    exe = str(tmp_path / "dinr_example")
    cmd = ["gcc", "-std=c11", "-O2", "-Wall", "-Wextra", "-Werror", SRC,
           "-I", os.path.join(ROOT, "include"), "-L", LIBDIR, "-ldinr",
           f"-Wl,-rpath,{LIBDIR}", "-lm", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_example_builds(tmp_path):
    assert os.path.exists(_build(tmp_path))


@pytest.mark.gpu
def test_c_example_trains(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    exe = _build(tmp_path)
    r = subprocess.run([exe, "300"], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "loss" in r.stdout
