"""The Fourier-slice projector's target geometry on the host: a program
(tests/c_abi/slice_taps.cu) built with nvcc against the library's internal
header checks, for every accepted angle count up to 1024 and every grid size,
that every tap of every target falls inside the stored half grid and its tile
(the kernels read shared memory there without a bounds check), and that the
wrapped and folded targets of half-size images sit at y = -j e modulo the
grid period (T(-s) = conj T(s) when folded); and a second program
(tests/c_abi/slice_groups.cu) builds the interpolation's target tables with
the library's host code (sw_slice_plan.h) and checks that every target is
covered exactly once, that every pair entry is one the kernel can take
without a check, and the half-warp grouping the kernel's speed relies on;
a third (tests/c_abi/slice_kernel.cu) checks the spreading kernel's host-side
numbers (tap-weight polynomials, Fourier transform) against FP64 references
and the accuracy of a 1-D type-2 NUFFT made of them.  Host code only: no
device."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _build_and_run(tmp_path, name):
    nvcc = os.path.join(CUDA, "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if not nvcc:
        pytest.skip("no nvcc")
    exe = str(tmp_path / name)
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-x", "cu",
                        "-I", os.path.join(ROOT, "paper_2503_13756_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "c_abi", name + ".cu"), "-o", exe],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout


def test_every_tap_inside_the_stored_grid(tmp_path):
    out = _build_and_run(tmp_path, "slice_taps")
    assert out.startswith("ok"), out


def test_target_tables_cover_every_target_once(tmp_path):
    out = _build_and_run(tmp_path, "slice_groups")
    assert out.rstrip().endswith("ok"), out


def test_spreading_kernel_numbers_and_nufft_accuracy(tmp_path):
    # tap-weight polynomials against the kernel, its Fourier transform against
    # quadrature, and a 1-D type-2 NUFFT of these parts against the direct sum
    out = _build_and_run(tmp_path, "slice_kernel")
    assert out.rstrip().endswith("ok"), out
