"""Host logic of the serving loop's admission (no GPU): the batch is formed
from the head of the FIFO, whole requests while they fit the batch limit, a
larger request split with its rest left at the head, the count halved while
the batch's workspace would exceed the slot's memory budget, and an empty
batch always taking at least one image so that the queue drains."""
import collections
import threading

import numpy as np

from paper_2503_13756_gb300 import serving


class StubBank:
    """workspace_bytes(Nq, mode): a fixed cost per query image."""

    def __init__(self, per_image, base=0):
        self.per_image, self.base = per_image, base

    def workspace_bytes(self, nq, mode):
        return self.base + self.per_image * nq


def engine(max_batch, budget, per_image, sizes):
    e = object.__new__(serving.ServingEngine)  # admission state only
    e.lock = threading.Lock()
    e.max_batch = max_batch
    e.slot_budget = budget
    e.bank = StubBank(per_image)
    e.queue = collections.deque()
    for rid, count in enumerate(sizes):
        req = serving.Request(rid=rid, images=np.zeros((count, 4, 4), np.float32))
        e.queue.append((req, 0))
    return e


def drain(e):
    batches = []
    while e.queue:
        batch, used = e._form_batch()
        assert used == sum(c for _, _, c in batch) and used > 0
        batches.append([(r.rid, s0, c) for r, s0, c in batch])
    return batches


def test_whole_requests_while_they_fit_then_a_split():
    e = engine(max_batch=10, budget=10 ** 9, per_image=1, sizes=[3, 4, 6, 2])
    assert drain(e) == [[(0, 0, 3), (1, 0, 4), (2, 0, 3)], [(2, 3, 3), (3, 0, 2)]]


def test_every_image_is_taken_once_in_fifo_order():
    rng = np.random.default_rng(3)
    sizes = list(rng.integers(1, 40, size=25))
    e = engine(max_batch=17, budget=10 ** 9, per_image=1, sizes=sizes)
    seen = []
    for b in drain(e):
        assert sum(c for _, _, c in b) <= 17
        for rid, s0, c in b:
            seen.extend((rid, k) for k in range(s0, s0 + c))
    assert seen == [(rid, k) for rid, n in enumerate(sizes) for k in range(n)]


def test_memory_budget_halves_the_count():
    # budget for 5 images: the 12-image request is cut 12 -> 6 -> 3, then its
    # rest (now at the head) tops the batch up to the budget, 9 -> 4 -> 2
    e = engine(max_batch=64, budget=5, per_image=1, sizes=[12])
    batches = drain(e)
    assert all(sum(c for _, _, c in b) <= 5 for b in batches)
    assert sum(c for b in batches for _, _, c in b) == 12
    assert batches[0] == [(0, 0, 3), (0, 3, 2)]


def test_a_second_request_waits_when_it_would_break_the_budget():
    e = engine(max_batch=64, budget=6, per_image=1, sizes=[4, 4])
    assert drain(e) == [[(0, 0, 4), (1, 0, 2)], [(1, 2, 2)]]


def test_budget_below_one_image_still_drains_one_at_a_time():
    e = engine(max_batch=64, budget=0, per_image=1, sizes=[3, 2])
    assert drain(e) == [[(0, 0, 1)], [(0, 1, 1)], [(0, 2, 1)], [(1, 0, 1)], [(1, 1, 1)]]
