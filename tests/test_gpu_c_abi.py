"""The C ABI from plain C: a C program (tests/c_abi/align_pair.c), compiled
with gcc against include/swalign.h and linked to the library, scores one pair
at every rotation through sw_align_all_rotations; its printed curve, shifts
and argmin record match the oracle (Eq. discrete_rot_sw2 with the closed-form
translation of Sec. 2.2) within the FP32 bar.  No Python binding sits on
this path.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2503_13756_gb300 import build, synth
from tests.parity import check_argmin, d2_tol, norm_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def compile_program(tmp_path):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    lib = build.build()
    exe = str(tmp_path / "align_pair")
    libdir = os.path.dirname(lib)
    cudalib = os.path.join(CUDA, "lib64")
    cmd = [gcc, "-std=c11", "-O2", "-Wall", "-Werror",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           os.path.join(ROOT, "tests", "c_abi", "align_pair.c"), "-o", exe,
           "-L", libdir, "-lswalign", "-L", cudalib, "-lcudart",
           f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{cudalib}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def test_c_program_matches_oracle(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = compile_program(tmp_path)
    L, n, M = 48, 72, 40
    rng = np.random.default_rng(2024)
    imgs = synth.render(synth.draw_mixtures(rng, 2, L, ncomp=(2, 4)), L).astype(np.float32)
    path = tmp_path / "pair.f32"
    np.ascontiguousarray(imgs).tofile(path)
    r = subprocess.run([exe, str(path), str(L), str(n), str(M)], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = r.stdout.strip().splitlines()
    head = lines[0].split()
    assert head[0] == "best_l" and head[2] == "status" and head[4] == "shift" and head[7] == "d2"
    best_l, status = int(head[1]), int(head[3])
    shift = np.array([float(head[5]), float(head[6])])
    d2 = float(head[8])
    curve = np.array([[float(x) for x in ln.split()] for ln in lines[1:]])
    assert curve.shape == (n, 3)

    f, g = imgs[0].astype(np.float64), imgs[1].astype(np.float64)
    ref, Dref, Sref = oracle.align_pair(f, g, n, M, translation=1)
    Sc = norm_scale(f, g, n, M)
    tol = d2_tol(Dref, Sc)
    assert np.all(np.abs(curve[:, 0] - Dref) <= tol), np.max(np.abs(curve[:, 0] - Dref) / tol)
    np.testing.assert_allclose(curve[:, 1:], Sref, rtol=0, atol=1e-6)
    assert status == 0
    assert check_argmin(best_l, ref["best_l"], Dref, d2_tol(ref["d2"], Sc))
    assert abs(d2 - Dref[best_l]) <= d2_tol(Dref[best_l], Sc)
    np.testing.assert_allclose(shift, Sref[best_l], rtol=0, atol=1e-6)
