"""The multi-rank path of the benchmark on CPU: two gloo ranks.

Pairs are independent, so N GPUs run either N replicas of the workload (weak
scaling) or one workload with its query rows split over the ranks and the
templates replicated (strong scaling), with no data exchange; the only
cross-rank steps are the barrier around the timed region, the maximum of the
per-rank step times and the sum of the pairs processed.
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
    rank r's workload with bench.rank_seed(r)), so no two replicas repeat
    each other's pairs."""
    import numpy as np

    import bench
    from paper_2503_13756_gb300 import synth
    assert bench.rank_seed(0) != bench.rank_seed(1)
    a = synth.many_to_many(n_queries=4, n_templates=2, seed=bench.rank_seed(0))
    b = synth.many_to_many(n_queries=4, n_templates=2, seed=bench.rank_seed(1))
    a2 = synth.many_to_many(n_queries=4, n_templates=2, seed=bench.rank_seed(0))
    assert not np.array_equal(a["queries"], b["queries"])
    assert not np.array_equal(a["templates"], b["templates"])
    assert np.array_equal(a["queries"], a2["queries"])


def test_row_blocks_cover_every_query_once():
    import bench
    for nq in (0, 1, 7, 4096, 4097):
        for world in (1, 2, 3, 8):
            blocks = [bench.row_block(nq, world, r) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == nq
            for (a, b), (c, d) in zip(blocks, blocks[1:]):
                assert b == c
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1


def _row_worker(rank, world, port, q):
    # strong scaling: one workload, rank r scores its query rows against every
    # template (here with the FP64 oracle, the CPU stand-in for the kernels),
    # and the row blocks are gathered on every rank
    import numpy as np

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_2503_13756_gb300 import synth
    d = synth.many_to_many(n_queries=7, n_templates=3, L=16, seed=bench.rank_seed(0))
    lo, hi = bench.row_block(7, world, rank)
    part = oracle.align_all_pairs(d["queries"][lo:hi], d["templates"], 8, 6, nthreads=1)
    parts = [None] * world
    dist.all_gather_object(parts, (lo, hi, part))
    q.put((rank, parts))
    dist.destroy_process_group()


def test_row_partition_union_equals_one_full_run():
    import numpy as np

    import bench
    import oracle
    from paper_2503_13756_gb300 import synth
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_row_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    d = synth.many_to_many(n_queries=7, n_templates=3, L=16, seed=bench.rank_seed(0))
    full = oracle.align_all_pairs(d["queries"], d["templates"], 8, 6, nthreads=1)
    for rank, parts in out:
        rows = np.concatenate([part for lo, hi, part in sorted(parts, key=lambda x: x[0])])
        assert [(lo, hi) for lo, hi, _ in parts] == [bench.row_block(7, world, r)
                                                     for r in range(world)]
        np.testing.assert_array_equal(rows, full)
