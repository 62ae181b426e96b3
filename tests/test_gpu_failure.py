"""Failure detection on the GPU without a fault (the tensor-core
correlation's bounded pipeline waits).

The correlation kernel's roles (TMA producer, MMA issuer, epilogue) wait on
one another through mbarriers; every such wait gives up after a limit
(sw_set_wait_limit), stops the kernel's remaining work once the copies and
MMAs already issued have landed, and turns every result of the call into
status 3 with NaN values.  The test makes a wait run out on purpose: with
the stall hook on, the producer issues no copies, so the MMA role waits on a
barrier that nothing completes.  The call still returns, the context stays
usable, and the next call gives the normal results bit for bit.
"""
import numpy as np
import pytest

from paper_2503_13756_gb300 import swalign, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def al():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    a = swalign.Aligner(0)
    yield a
    a.set_correlation_stall(False)
    a.set_wait_limit(0)
    a.close()


@pytest.mark.parametrize("precision,projector", [("fp32", "slice"), ("bf16", "splat")])
def test_wait_that_runs_out_gives_status_3_and_the_context_recovers(al, precision, projector):
    rng = np.random.default_rng(404)
    L, n, M = 32, 24, 16
    q = synth.render(synth.draw_mixtures(rng, 40, L, ncomp=(2, 3)), L).astype(np.float32)
    t = synth.render(synth.draw_mixtures(rng, 9, L, ncomp=(2, 3)), L).astype(np.float32)
    p = swalign.make_params(L, n, M, precision=precision, projector=projector)
    ref = swalign.results_to_numpy(al.align_batch(q, t, p))
    assert np.all(ref["status"] == 0)
    al.set_wait_limit(2_000_000)  # ~1 ms of SM clock
    al.set_correlation_stall(True)
    try:
        bad = swalign.results_to_numpy(al.align_batch(q, t, p))
        bank = swalign.Bank(al, t, p)
        try:
            bad_bank = swalign.results_to_numpy(bank.align(q))
        finally:
            bank.close()
    finally:
        al.set_correlation_stall(False)
        al.set_wait_limit(0)
    torch.cuda.synchronize()  # the device is still usable
    for r in (bad, bad_bank):
        assert np.all(r["status"] == 3)
        assert np.all(np.isnan(r["d2"])) and np.all(r["best_l"] == -1)
    again = swalign.results_to_numpy(al.align_batch(q, t, p))
    np.testing.assert_array_equal(again["status"], ref["status"])
    np.testing.assert_array_equal(again["best_l"], ref["best_l"])
    np.testing.assert_array_equal(again["d2"], ref["d2"])


def test_wait_limit_arguments(al):
    with pytest.raises(swalign.SwError) as e:
        al.set_wait_limit(-1)
    assert e.value.status == swalign.SW_ERR_INVALID_ARG
    al.set_wait_limit(0)
