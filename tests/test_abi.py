"""CPU checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point that include/swalign.h declares.  No GPU call."""
import ctypes
import os
import re

import pytest

import oracle
from paper_2503_13756_gb300 import swalign

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "swalign.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sw_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("sw_project", "sw_quantiles", "sw_align_all_rotations", "sw_align_batch",
                 "sw_create", "sw_destroy", "sw_last_error", "sw_bank_create",
                 "sw_bank_align", "sw_bank_destroy"):
        assert name in syms


def test_library_exports_every_declared_symbol():
    lib = swalign.load()
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    assert set(swalign.EXPORTS) <= set(declared_symbols())


def test_result_struct_layout():
    # sw_result: int32 best_l, int32 status, float angle, int32 template_index,
    # double shift[2], double d2 -> 40 bytes, d2 at offset 32
    assert swalign.RESULT_DTYPE.itemsize == 40
    assert swalign.RESULT_DTYPE.fields["d2"][1] == 32
    assert ctypes.sizeof(swalign.Params) == 44


def test_params_fields_follow_the_header():
    with open(os.path.join(ROOT, "include", "swalign.h")) as fh:
        text = fh.read()
    body = text[text.index("typedef struct {\n    int32_t L;"):text.index("} sw_params;")]
    fields = re.findall(r"int32_t\s+(\w+);", body)
    assert fields == [f[0] for f in swalign.Params._fields_]


def test_default_bins_agree_with_oracle():
    lib = swalign.load()
    for L in [2, 3, 16, 39, 64, 85, 96, 128, 192, 256, 512]:
        assert lib.sw_default_bins(L) == oracle.default_bins(L)
        p = swalign.make_params(L, 8, 4, metric="rfsw2")
        assert swalign.bins_of(p) == oracle.rfsw_bins(L)
        p = swalign.make_params(L, 8, 4, projector="slice")
        assert swalign.bins_of(p) == oracle.bins_for(L, projector=1)


def test_workspace_size_is_host_computable():
    lib = swalign.load()
    p = swalign.make_params(128, 256, 128)
    small = lib.sw_batch_workspace_bytes(ctypes.byref(p), 16, 8)
    big = lib.sw_batch_workspace_bytes(ctypes.byref(p), 4096, 256)
    assert 0 < small < big
    bad = swalign.make_params(128, 257, 128)  # odd n is rejected
    assert lib.sw_batch_workspace_bytes(ctypes.byref(bad), 16, 8) == 0


def test_without_a_device_the_product_path_fails_loudly():
    """No CPU fallback: on a machine with no visible CUDA device the Python
    context raises and sw_create returns an error with no context."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is visible")
    with pytest.raises(RuntimeError):
        swalign.Aligner(0)
    lib = swalign.load()
    h = ctypes.c_void_p(1)
    assert lib.sw_create(0, ctypes.byref(h)) != 0
    assert not h.value
    assert lib.sw_create(0, None) == 1  # SW_ERR_INVALID_ARG


def test_build_targets_sm_103a_only_and_compiles_every_source():
    from paper_2503_13756_gb300 import build as b
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert "-lineinfo" in b.NVCC_FLAGS and "-O3" in b.NVCC_FLAGS
    flags = " ".join(b.NVCC_FLAGS)
    assert "march" not in flags and "sm_90" not in flags and "sm_100" not in flags
    names = sorted(os.path.basename(s) for s in b.sources())
    on_disk = sorted(f for f in os.listdir(b.CSRC) if f.endswith(".cu"))
    assert names == on_disk and "sw_api.cu" in names
    assert os.path.exists(b.build())
