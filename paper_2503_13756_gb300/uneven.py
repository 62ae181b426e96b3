"""Uneven batches as one CUDA graph.

An uneven batch holds queries of several sizes L, each size scored against
its own templates (n_theta angles, M levels, a GEMM precision per size).
Every size is one sw_align_batch call; the calls of all sizes are captured
once into a CUDA graph, and each later batch of the same shapes is one graph
launch: no per-kernel host work, no Python between the sizes.  By default
every size has its own context (workspace) and stream, forked from and
joined back into the graph's stream, so the sizes are independent branches
of the graph and their kernels overlap where the GPU has room (a
latency-bound stage of one size beside a busy stage of another);
concurrent=False captures them back to back on one stream with one context.

Capture needs a call that allocates nothing and synchronises nothing: the
context's workspace is reserved for the largest size first (sw_reserve, which
also builds the angle tables), the launch shapes are autotuned (optional)
and the whole batch is run once eagerly before capture, so that every
one-time setup (kernel attributes, the tensor-map encoder) is done.  Inputs
and outputs are fixed device buffers: refill the inputs in place and replay.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import swalign


@dataclass
class Bucket:
    L: int
    params: swalign.Params
    queries: "object"    # torch.Tensor [Nq][L][L] float32 on the device
    templates: "object"  # torch.Tensor [Nt][L][L] float32 on the device
    out: "object" = None  # torch.Tensor [rows][40] uint8 (sw_result rows)


class UnevenGraph:
    """Scores every bucket (mode 0: all pairs [Nq][Nt]; mode 1: best
    template per query) in one graph launch."""

    def __init__(self, buckets, mode: int = 0, device: int = 0, autotune: bool = False,
                 cache_path: str | None = None, concurrent: bool = True):
        import torch
        self.torch = torch
        self.device = device
        self.mode = mode
        self.concurrent = concurrent
        # the largest sizes first: their branches start first
        self.buckets = sorted(buckets, key=lambda b: -b.L) if concurrent else list(buckets)
        n_ctx = len(self.buckets) if concurrent else 1
        self.als = [swalign.Aligner(device) for _ in range(max(1, n_ctx))]
        self.al = self.als[0]
        for i, b in enumerate(self.buckets):
            Nq, Nt = b.queries.shape[0], b.templates.shape[0]
            rows = Nq * Nt if mode == 0 else Nq
            if b.out is None:
                b.out = torch.empty((rows, 40), dtype=torch.uint8, device=b.queries.device)
            al = self._al(i)
            if autotune:
                al.autotune(b.params, cache_path)
            # a context's workspace grows to the largest size it runs
            al.reserve(b.params, Nq, Nt)
        self.stream = torch.cuda.Stream(device=device)
        self.branch = [torch.cuda.Stream(device=device) for _ in self.buckets] if concurrent \
            else []
        self.fork = torch.cuda.Event()
        self.join = [torch.cuda.Event() for _ in self.branch]
        with torch.cuda.stream(self.stream):
            self._run_all()  # eager pass: one-time setup happens outside the capture
        self.stream.synchronize()
        self.launches_per_replay = -self.launch_count()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream, capture_error_mode="thread_local"):
            self._run_all()
        self.launches_per_replay += self.launch_count()

    def _al(self, i):
        return self.als[i] if self.concurrent else self.als[0]

    def launch_count(self) -> int:
        return sum(a.launch_count() for a in self.als)

    def _run_all(self):
        """Every size once on the current stream: forked into one branch per
        size and joined back (concurrent), or back to back."""
        main = self.torch.cuda.current_stream()
        if not self.concurrent:
            for b in self.buckets:
                self.al.align_batch(b.queries, b.templates, b.params, mode=self.mode, out=b.out,
                                    stream=main)
            return
        self.fork.record(main)
        for i, b in enumerate(self.buckets):
            st = self.branch[i]
            st.wait_event(self.fork)
            with self.torch.cuda.stream(st):
                self.als[i].align_batch(b.queries, b.templates, b.params, mode=self.mode,
                                        out=b.out, stream=st)
            self.join[i].record(st)
        for ev in self.join:
            main.wait_event(ev)

    def replay(self):
        """Runs every bucket once (asynchronously, on the graph's stream,
        after the work already queued on the caller's current stream, such as
        a refill of the inputs)."""
        self.stream.wait_stream(self.torch.cuda.current_stream())
        with self.torch.cuda.stream(self.stream):
            self.graph.replay()

    def stage_times(self):
        """Milliseconds per stage for every size, from one eager pass with
        the kernel events of the profiler (waits for the device)."""
        out = {}
        self.stream.synchronize()
        for i, b in enumerate(self.buckets):
            al = self._al(i)
            al.profile(True)
            al.profile_read()
            try:
                with self.torch.cuda.stream(self.stream):
                    al.align_batch(b.queries, b.templates, b.params, mode=self.mode,
                                   out=b.out, stream=self.stream)
                    out[b.L] = {k: v[0] for k, v in al.profile_read().items()}
            finally:
                al.profile(False)
        return out

    def run_eager(self):
        """The same calls without the graph (for comparison)."""
        self.stream.wait_stream(self.torch.cuda.current_stream())
        with self.torch.cuda.stream(self.stream):
            self._run_all()

    def results(self):
        """Structured results per bucket, keyed by L (waits for the device)."""
        self.stream.synchronize()
        return {b.L: swalign.results_to_numpy(b.out) for b in self.buckets}

    @property
    def pairs(self) -> int:
        return sum(b.queries.shape[0] * b.templates.shape[0] for b in self.buckets)

    def close(self):
        self.graph = None
        for a in self.als:
            a.close()


def buckets_from(batch, n_theta: int = 256, precision: str = "bf16", device: int = 0,
                 projector: str = "splat"):
    """Device buckets from a host batch {L: {"queries", "templates"}} with
    M = L levels per size (the uneven-batch recipe)."""
    import torch
    out = []
    for L in sorted(batch):
        d = batch[L]
        q = torch.as_tensor(d["queries"], dtype=torch.float32).to(f"cuda:{device}")
        t = torch.as_tensor(d["templates"], dtype=torch.float32).to(f"cuda:{device}")
        out.append(Bucket(L, swalign.make_params(L, n_theta, L, precision=precision,
                                                 projector=projector), q, t))
    return out
