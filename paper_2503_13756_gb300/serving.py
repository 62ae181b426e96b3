"""Serving loop: continuous batching of alignment requests against a
device-resident template bank.

Each request carries a few query images (at the bank's side L, or L/2, which
the library upsamples 2 x 2 on load).  For every query the server returns the
best template of the bank with its rotation, translation and squared sliced-W2
distance (sw_bank_align, mode 1).

Design: requests wait in a FIFO.  The engine owns several slots, each a CUDA
stream with its own library context (and so its own workspace), pinned host
staging buffers and device buffers.  Whenever a slot is free and requests are
waiting, a batch is formed from the head of the queue -- whole requests while
they fit, splitting a request that is larger than the batch limit -- subject to
memory-based admission: the batch's workspace (sw_bank_workspace_bytes) must
fit the slot's share of the device memory that was free at start-up.  A batch
is launched (copy in, one sw_bank_align per image size, copy out, event) and
the loop goes back to admitting, so requests that arrive while others are on
the GPU join the next batch and their work overlaps on the device.  A request
completes when the host has the results of all its images; its latency is
measured from its arrival to that moment.

Results do not depend on which batch a query lands in beyond rounding: every
query-template pair is computed from its own spectra with a fixed reduction
order; only the decision FFT, which packs two pairs per complex signal, lets a
neighbouring pair's values enter the rounding.
"""
from __future__ import annotations

import collections
import gc
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import swalign


@dataclass
class Request:
    rid: int
    images: np.ndarray            # [count][Lq][Lq] float32
    t_arrive: float = 0.0         # seconds from the start of the run
    t_done: float = -1.0
    results: np.ndarray = None    # structured RESULT_DTYPE [count]
    remaining: int = 0
    _t_arrive_abs: float = field(default=0.0, repr=False)


def make_requests(pool, schedule):
    """Requests from a pool of images per size ({L: {"images", "source"}}) and a
    schedule (arrival times, counts, sizes, pick indices)."""
    t, counts, Ls, picks = schedule
    reqs = []
    for r in range(len(t)):
        P = pool[int(Ls[r])]
        idx = np.asarray(picks[r]) % len(P["images"])
        req = Request(rid=r, images=np.ascontiguousarray(P["images"][idx]), t_arrive=float(t[r]))
        req.source = P["source"][idx]
        reqs.append(req)
    return reqs


class _Slot:
    def __init__(self, device, L, max_images, Nt):
        import torch
        self.al = swalign.Aligner(device)
        self.stream = torch.cuda.Stream(device=device)
        self.L = L
        self.h_full = torch.empty((max_images, L, L), dtype=torch.float32).pin_memory()
        self.h_half = torch.empty((max_images, L // 2, L // 2), dtype=torch.float32).pin_memory()
        self.d_full = torch.empty((max_images, L, L), dtype=torch.float32, device=device)
        self.d_half = torch.empty((max_images, L // 2, L // 2), dtype=torch.float32, device=device)
        self.d_out = torch.empty((max_images, 40), dtype=torch.uint8, device=device)
        self.h_out = torch.empty((max_images, 40), dtype=torch.uint8).pin_memory()
        self.event = torch.cuda.Event()
        self.batch = None  # list of (request, start, count, row) while in flight

    def close(self):
        self.al.close()


class ServingEngine:
    """Continuous-batching front end of sw_bank_align.  The defaults (six
    slots, at most 128 images per batch) split a large request across slots
    so that its parts run concurrently; against a 1000-template bank of 256^2
    they gave a lower p99 than three slots of 512 images, for 5% less
    throughput at saturation."""

    def __init__(self, templates, params: swalign.Params, n_slots: int = 6,
                 max_batch_images: int = 128, device: int = 0, mem_fraction: float = 0.5,
                 autotune: bool = False):
        import torch
        torch.cuda.set_device(device)
        self.device = device
        self.params = params
        self.L = params.L
        self.main = swalign.Aligner(device)
        if autotune:  # the bank keeps the launch shapes in force at its creation
            self.main.autotune(params)
        self.bank = swalign.Bank(self.main, templates, params)
        self.Nt = self.bank.Nt
        free, _ = torch.cuda.mem_get_info(device)
        self.slot_budget = int(free * mem_fraction / max(1, n_slots))
        # largest batch whose workspace fits a slot's share (memory-based admission)
        mb = max_batch_images
        while mb > 1 and self.bank.workspace_bytes(mb, 1) > self.slot_budget:
            mb //= 2
        self.max_batch = mb
        self.slots = [_Slot(device, self.L, mb, self.Nt) for _ in range(n_slots)]
        for s in self.slots:
            # size each slot's workspace and run both query sizes once (tables,
            # kernel attributes, first launches), outside the timed loop
            s.d_full.zero_()
            s.d_half.zero_()
            self.bank.align(s.d_full[:mb], q_L=self.L, mode=1, out=s.d_out[:mb],
                            stream=s.stream, aligner=s.al)
            if self.L % 2 == 0:
                self.bank.align(s.d_half[:mb], q_L=self.L // 2, mode=1, out=s.d_out[:mb],
                                stream=s.stream, aligner=s.al)
        torch.cuda.synchronize()
        self.queue = collections.deque()
        self.lock = threading.Lock()
        self.batches = 0
        self.batch_sizes = []

    def close(self):
        for s in self.slots:
            s.close()
        self.bank.close()
        self.main.close()

    # ------------------------------------------------------------ admission
    def _form_batch(self):
        """Whole requests from the queue head while they fit; a request larger
        than what is left is split and its rest stays at the head."""
        batch, used = [], 0
        with self.lock:
            while self.queue and used < self.max_batch:
                req, start = self.queue[0]
                take = min(len(req.images) - start, self.max_batch - used)
                # shrink to the budget; an empty batch always takes one image,
                # so that the queue drains even under a budget below one image
                while take > 1 and self.bank.workspace_bytes(used + take, 1) > self.slot_budget:
                    take //= 2
                if used and self.bank.workspace_bytes(used + take, 1) > self.slot_budget:
                    break
                batch.append((req, start, take))
                used += take
                if start + take == len(req.images):
                    self.queue.popleft()
                else:
                    self.queue[0] = (req, start + take)
        return batch, used

    def _launch(self, slot, batch):
        import torch
        full = [(r, s0, c) for (r, s0, c) in batch if r.images.shape[-1] == self.L]
        half = [(r, s0, c) for (r, s0, c) in batch if r.images.shape[-1] != self.L]
        placed, row = [], 0
        nf = nh = 0
        for group, h_buf in ((full, slot.h_full), (half, slot.h_half)):
            k = 0
            for (r, s0, c) in group:
                h_buf[k:k + c].copy_(torch.from_numpy(r.images[s0:s0 + c]))
                placed.append((r, s0, c, row))
                row += c
                k += c
            if group is full:
                nf = k
            else:
                nh = k
        with torch.cuda.stream(slot.stream):
            if nf:
                slot.d_full[:nf].copy_(slot.h_full[:nf], non_blocking=True)
                self.bank.align(slot.d_full[:nf], q_L=self.L, mode=1, out=slot.d_out[:nf],
                                stream=slot.stream, aligner=slot.al)
            if nh:
                slot.d_half[:nh].copy_(slot.h_half[:nh], non_blocking=True)
                self.bank.align(slot.d_half[:nh], q_L=self.L // 2, mode=1,
                                out=slot.d_out[nf:nf + nh], stream=slot.stream, aligner=slot.al)
            slot.h_out[:nf + nh].copy_(slot.d_out[:nf + nh], non_blocking=True)
            slot.event.record(slot.stream)
        slot.batch = placed
        self.batches += 1
        self.batch_sizes.append(nf + nh)

    def _harvest(self, slot, t0):
        res = swalign.results_to_numpy(slot.h_out[:sum(c for _, _, c, _ in slot.batch)])
        now = time.perf_counter() - t0
        for (r, s0, c, row) in slot.batch:
            r.results[s0:s0 + c] = res[row:row + c]
            r.remaining -= c
            if r.remaining == 0:
                r.t_done = now
        slot.batch = None

    # ----------------------------------------------------------------- run
    def run(self, requests, realtime: bool = True):
        """Feeds the requests at their arrival times (realtime) or all at
        once, serves them, and returns summary statistics.  The interpreter's
        cyclic garbage collector is paused while the loop runs (reference
        counting still frees every object; a collection pass over a large heap
        would stall the loop for milliseconds) and restored on return."""
        was_enabled = gc.isenabled()
        gc.disable()
        try:
            return self._run(requests, realtime)
        finally:
            if was_enabled:
                gc.enable()

    def _run(self, requests, realtime):
        for r in requests:
            r.results = np.zeros(len(r.images), dtype=swalign.RESULT_DTYPE)
            r.remaining = len(r.images)
            r.t_done = -1.0
        pending = sorted(requests, key=lambda r: r.t_arrive)
        t0 = time.perf_counter()
        i_next = 0
        done = 0
        while done < len(requests):
            now = time.perf_counter() - t0
            while i_next < len(pending) and (not realtime or pending[i_next].t_arrive <= now):
                r = pending[i_next]
                if not realtime:
                    r.t_arrive = now
                with self.lock:
                    self.queue.append((r, 0))
                i_next += 1
            progressed = False
            for s in self.slots:
                if s.batch is not None and s.event.query():
                    before = sum(1 for r in requests if r.t_done >= 0)
                    self._harvest(s, t0)
                    done += sum(1 for r in requests if r.t_done >= 0) - before
                    progressed = True
            for s in self.slots:
                if s.batch is None and self.queue:
                    batch, used = self._form_batch()
                    if used:
                        self._launch(s, batch)
                        progressed = True
            if not progressed:
                time.sleep(50e-6)
        wall = time.perf_counter() - t0
        lat = np.array([r.t_done - r.t_arrive for r in requests])
        images = sum(len(r.images) for r in requests)
        return {
            "requests": len(requests), "images": images, "pairs": images * self.Nt,
            "wall_s": wall, "pairs_per_s": images * self.Nt / wall,
            "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)),
                           "p99": 1e3 * float(np.percentile(lat, 99)),
                           "max": 1e3 * float(lat.max())},
            "batches": self.batches,
            "mean_batch_images": float(np.mean(self.batch_sizes)) if self.batch_sizes else 0.0,
            "max_batch_images": self.max_batch,
        }
