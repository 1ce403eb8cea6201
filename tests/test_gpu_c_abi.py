"""The C ABI from a plain C99 program (tests/c_abi_track.c): built with gcc
against include/phd.h, linked to libphd.so and the CUDA runtime, run on the
GPU; it tracks two targets through phd_step and phd_step_host."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def build_c_program(out):
    pkg = os.path.join(ROOT, "paper_1503_03769_gb300")
    cmd = ["gcc", "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(CUDA, "include"), os.path.join(ROOT, "tests", "c_abi_track.c"), "-o", out,
           "-L", pkg, "-lphd", "-Wl,-rpath," + pkg, "-L", os.path.join(CUDA, "lib64"), "-lcudart",
           "-Wl,-rpath," + os.path.join(CUDA, "lib64"), "-lm"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)


@pytest.mark.gpu
def test_c_program_tracks_through_the_c_abi(tmp_path):
    exe = str(tmp_path / "track")
    build_c_program(exe)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "tracked" in r.stdout and ": ok" in r.stdout, r.stdout
