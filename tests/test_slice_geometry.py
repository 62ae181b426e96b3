"""The Fourier-slice projector's target geometry on the host: a program
(tests/c_abi/slice_taps.cu) built with nvcc against the library's internal
header checks, for every accepted angle count up to 1024 and every grid size,
that every tap of every target falls inside the stored half grid and its tile
(the kernels read shared memory there without a bounds check), and that the
wrapped and folded targets of half-size images sit at y = -j e modulo the
grid period (T(-s) = conj T(s) when folded).  Host code only: no device."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def test_every_tap_inside_the_stored_grid(tmp_path):
    nvcc = os.path.join(CUDA, "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if not nvcc:
        pytest.skip("no nvcc")
    exe = str(tmp_path / "slice_taps")
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-x", "cu",
                        "-I", os.path.join(ROOT, "paper_2503_13756_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "c_abi", "slice_taps.cu"), "-o", exe],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
