"""The CUDA path against the stored oracle values of tests/golden/
golden_cases.json (single pair through sw_align_all_rotations; quantiles
through sw_project + sw_quantiles), at the FP32 parity bar."""
import numpy as np
import pytest

from paper_2503_13756_gb300 import swalign
from tests.parity import check_argmin, d2_tol, norm_scale, q_tol
from tests.test_golden import golden_cases

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def al():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    a = swalign.Aligner(0)
    yield a
    a.close()


@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: c["name"])
def test_gpu_matches_golden_case(al, case):
    f = np.array(case["f"], dtype=np.float32)
    g = np.array(case["g"], dtype=np.float32)
    n, M, L = case["n"], case["M"], case["L"]
    p = swalign.make_params(L, n, M, translation=case["translation"],
                            level_rule=case["level_rule"])
    D, S, best = al.align_all_rotations(f, g, p)
    D, S = D.cpu().numpy(), S.cpu().numpy()
    Dref, Sref = np.array(case["D"]), np.array(case["shifts"])
    Sc = norm_scale(f.astype(np.float64), g.astype(np.float64), n, M, case["level_rule"])
    assert np.all(np.abs(D - Dref) <= d2_tol(Dref, Sc))
    np.testing.assert_allclose(S, Sref, rtol=0, atol=1e-6)
    r = swalign.results_to_numpy(best)[0]
    assert check_argmin(int(r["best_l"]), case["best_l"], Dref, d2_tol(case["d2"], Sc))
    proj = al.project(f[None], p)
    Q, _, _ = al.quantiles(proj, p)
    Qref = np.array(case["quantiles_f"])
    assert np.all(np.abs(Q.cpu().numpy()[0] - Qref) <= q_tol(Qref))
