"""The benchmark's measured-error report (the `parity` key) on the CPU: the
metrics of parity_of on constructed results, and the oracle leg of
cpu_baseline on a tiny workload scored against the oracle's own results."""
import numpy as np

import bench
import oracle
from paper_2503_13756_gb300 import synth


def _results(d2, best_l, shift=0.0):
    r = np.zeros(len(d2), dtype=oracle.RESULT_DTYPE)
    r["d2"] = d2
    r["best_l"] = best_l
    r["shift"] = shift
    return r


def test_parity_of_reports_plain_and_floored_errors():
    ref = _results([1e-4, 1e-2, 5e-2], [3, 10, 200])
    gpu = _results([1e-4 * (1 + 2e-3), 1e-2 * (1 + 1e-6), 5e-2], [3, 11, 200], shift=1e-7)
    S = np.array([0.2, 0.2, 0.2])
    p = bench.parity_of(gpu, ref, S, 1e-5)
    assert p["pairs"] == 3
    assert abs(p["max_rel_d2"] - 2e-3) < 1e-12
    assert abs(p["argmin_same"] - 2 / 3) < 1e-12 and p["argmin_within_1_bin"] == 1.0
    assert abs(p["frac_rel_d2_above_1e-5"] - 1 / 3) < 1e-12
    # the bar 1e-5 max(d2, 0.1 S) at d2 = 1e-4, S = 0.2 is 2e-7 (+ 1e-12)
    assert abs(p["worst_ratio_to_bar"] - 2e-7 / (2e-7 + 1e-12)) < 1e-6
    assert abs(p["max_abs_d2_over_S"] - 2e-7 / 0.2) < 1e-15
    assert abs(p["max_shift_err"] - 1e-7) < 1e-15
    assert abs(p["min_d2_over_S"] - 5e-4) < 1e-15


def test_cpu_baseline_scores_a_tiny_workload_against_itself():
    d = synth.many_to_many(n_queries=3, n_templates=2, L=16)
    s = 2
    q, t = d["queries"][:s], d["templates"][:s]
    ref = oracle.align_all_pairs(q.astype(np.float64), t.astype(np.float64), bench.N_THETA,
                                 bench.M_LEVELS, nthreads=1)
    src = d["source"][:s]
    ref_src = oracle.align_all_pairs(q.astype(np.float64), d["templates"][src].astype(np.float64),
                                     bench.N_THETA, bench.M_LEVELS, nthreads=1)[np.arange(s), np.arange(s)]
    norms = (np.ones(s), np.ones(s), np.ones(s))
    cpu, parity = bench.cpu_baseline(d, "splat", {"fp32": (ref, ref_src)}, norms, s)
    assert cpu["kind"] == "oracle" and cpu["value"] > 0
    for part in ("block", "source_pairs"):
        r = parity["fp32"][part]
        assert r["max_rel_d2"] == 0.0 and r["argmin_same"] == 1.0 and r["worst_ratio_to_bar"] == 0.0
    assert parity["fp32"]["block"]["pairs"] == s * s and parity["fp32"]["source_pairs"]["pairs"] == s
