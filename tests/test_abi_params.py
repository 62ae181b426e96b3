"""CPU checks of the parameter limits that include/swalign.h states for
sw_params.  sw_batch_workspace_bytes validates its parameters on the host
and returns 0 for an invalid set, so every limit can be checked without a
GPU: each value just outside a stated range is rejected, the edges and the
documented special cases are accepted."""
import ctypes

import pytest

from paper_2503_13756_gb300 import swalign


def ws_bytes(p, Nq=4, Nt=2):
    lib = swalign.load()
    return lib.sw_batch_workspace_bytes(ctypes.byref(p), Nq, Nt)


def with_(p, **fields):
    for k, v in fields.items():
        setattr(p, k, v)
    return p


def base(**kw):
    return swalign.make_params(64, 64, 32, **kw)


VALID = [
    ("L at its lower edge", with_(base(), L=2)),
    ("L at its upper edge", with_(base(), L=512)),
    ("n_theta = 4", with_(base(), n_theta=4)),
    ("n_theta = 1024", with_(base(), n_theta=1024)),
    ("n_theta with factors 2, 3, 5", with_(base(), n_theta=360)),
    ("n_levels = 1", with_(base(), n_levels=1)),
    ("n_levels = 1024", with_(base(), n_levels=1024)),
    ("n_bins at the default", with_(base(), n_bins=swalign.bins_of(base()))),
    ("n_bins = 2048", with_(base(), n_bins=2048)),
    ("rotation only", with_(base(), translation=0)),
    ("level rule p/M", with_(base(), level_rule=1)),
    ("BF16", base(precision="bf16")),
    ("FP16", base(precision="fp16")),
    ("FP32 on CUDA cores", base(precision="fp32_simt")),
    ("RFSW2 with 512 levels per part", with_(base(metric="rfsw2"), n_levels=512)),
    ("RFSW2 with a smooth bin count", with_(base(metric="rfsw2"), n_bins=96)),
    ("MSW2", base(metric="msw2")),
    ("translation grid", base(shift_grid=3, shift_step_q=8)),
    ("translation grid at its limits", base(shift_grid=4096, shift_step_q=65536)),
    ("slice projector, L = 128", swalign.make_params(128, 64, 32, projector="slice")),
    ("slice projector, L = 256", swalign.make_params(256, 64, 32, projector="slice")),
    ("slice projector, explicit 32 bins at L = 16",
     swalign.make_params(16, 64, 32, n_bins=32, projector="slice")),
    ("slice projector, 320 bins at L = 200",
     swalign.make_params(200, 64, 32, n_bins=320, projector="slice")),
]

INVALID = [
    ("L below 2", with_(base(), L=1)),
    ("L above 512", with_(base(), L=513)),
    ("odd n_theta", with_(base(), n_theta=63)),
    ("n_theta below 4", with_(base(), n_theta=2)),
    ("n_theta above 1024", with_(base(), n_theta=1026)),
    ("n_theta with a factor 7", with_(base(), n_theta=56)),
    ("n_levels = 0", with_(base(), n_levels=0)),
    ("n_levels above 1024", with_(base(), n_levels=1025)),
    ("n_bins below the default", with_(base(), n_bins=swalign.bins_of(base()) - 2)),
    ("odd n_bins", with_(base(), n_bins=swalign.bins_of(base()) + 1)),
    ("n_bins above 2048", with_(base(), n_bins=2050)),
    ("translation = 2", with_(base(), translation=2)),
    ("level_rule = 2", with_(base(), level_rule=2)),
    ("unknown precision", with_(base(), gemm_precision=4)),
    ("negative precision", with_(base(), gemm_precision=-1)),
    ("unknown metric", with_(base(), metric=3)),
    ("unknown projector", with_(base(), projector=2)),
    ("MSW2 with a translation grid", base(metric="msw2", shift_grid=2, shift_step_q=16)),
    ("negative shift grid", with_(base(), shift_grid=-1)),
    ("shift grid above 4096", base(shift_grid=4097, shift_step_q=16)),
    ("shift grid without a step", base(shift_grid=2, shift_step_q=0)),
    ("shift step above 65536", base(shift_grid=2, shift_step_q=65537)),
    ("RFSW2 with more than 512 levels", with_(base(metric="rfsw2"), n_levels=513)),
    ("RFSW2 with a bin count that is not 2/3/5-smooth",
     with_(base(metric="rfsw2"), n_bins=98)),
    ("slice projector above L = 256", swalign.make_params(288, 64, 32, projector="slice")),
    ("slice projector, bins not a multiple of 32",
     swalign.make_params(64, 64, 32, n_bins=112, projector="slice")),
    ("slice projector, bins below 1.5 L",
     swalign.make_params(100, 64, 32, n_bins=144, projector="slice")),
    ("slice projector, 288 bins above L = 128 (256, 320 or 384 only)",
     swalign.make_params(160, 64, 32, n_bins=288, projector="slice")),
    ("slice projector, 224 bins at L <= 128 (at most 192)",
     swalign.make_params(128, 64, 32, n_bins=224, projector="slice")),
]


@pytest.mark.parametrize("name,p", VALID, ids=[v[0] for v in VALID])
def test_documented_values_are_accepted(name, p):
    assert ws_bytes(p) > 0, name


@pytest.mark.parametrize("name,p", INVALID, ids=[v[0] for v in INVALID])
def test_values_outside_the_documented_ranges_are_rejected(name, p):
    assert ws_bytes(p) == 0, name


def test_negative_batch_sizes_and_null_params_are_rejected():
    p = base()
    assert ws_bytes(p, -1, 2) == 0
    assert ws_bytes(p, 4, -1) == 0
    lib = swalign.load()
    assert lib.sw_batch_workspace_bytes(None, 4, 2) == 0


def test_workspace_grows_with_the_batch():
    p = swalign.make_params(128, 256, 128, projector="slice")
    sizes = [ws_bytes(p, nq, 256) for nq in (256, 1024, 4096)]
    assert 0 < sizes[0] < sizes[1] < sizes[2]
    # the correlation output C (n/2 frequencies x Nq x Nt, complex FP32) and
    # the quantiles ([Nq + Nt][n][M] FP32) bound the workspace from below
    assert sizes[2] >= 8 * (256 // 2) * 4096 * 256 + 4 * (4096 + 256) * 256 * 128


def test_default_bins_of_the_slice_projector():
    """The slice projector's default bin count is the smallest multiple of
    32 that holds the default bins and 1.5 L; above L = 128 it is 256, 320
    or 384 (the grid lengths of the global-memory path)."""
    for L in range(2, 257):
        B = swalign.bins_of(swalign.make_params(L, 8, 4, projector="slice"))
        Bd = swalign.bins_of(swalign.make_params(L, 8, 4))
        assert B % 32 == 0 and B >= Bd and 2 * B >= 3 * L
        if L <= 128:
            assert B - 32 < max(Bd, (3 * L + 1) // 2)
        else:
            assert B in (256, 320, 384)
        assert ws_bytes(swalign.make_params(L, 8, 4, projector="slice")) > 0
