"""The multi-rank path of the benchmark on CPU: two gloo ranks.

Pairs are independent, so N GPUs run N replicas of the workload with no data
exchange; the only cross-rank steps are the barrier around the timed region,
the maximum of the per-rank step times and the sum of the pairs processed.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    cpu = torch.device("cpu")
    bench.barrier(world)
    ms = bench.max_over_ranks(10.0 + rank, world, cpu)       # slowest rank sets the time
    pairs = bench.sum_over_ranks(4096 * 256, world, cpu)      # every rank's pairs count
    q.put((rank, ms, pairs))
    dist.destroy_process_group()


def test_two_gloo_ranks_time_and_pairs():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, pairs in out:
        assert ms == 11.0
        assert pairs == world * 4096 * 256


def test_replicas_draw_distinct_inputs_per_rank():
    """Weak scaling: every rank aligns its own images (the benchmark seeds
    rank r's workload with SEED_BASE + 2 + 1000 r), so no two replicas
    repeat each other's pairs."""
    import numpy as np

    from paper_2503_13756_gb300 import synth
    a = synth.many_to_many(n_queries=4, n_templates=2, seed=synth.SEED_BASE + 2)
    b = synth.many_to_many(n_queries=4, n_templates=2, seed=synth.SEED_BASE + 2 + 1000)
    a2 = synth.many_to_many(n_queries=4, n_templates=2, seed=synth.SEED_BASE + 2)
    assert not np.array_equal(a["queries"], b["queries"])
    assert not np.array_equal(a["templates"], b["templates"])
    assert np.array_equal(a["queries"], a2["queries"])
