"""Uneven batches as one CUDA graph.

An uneven batch holds queries of several sizes L, each size scored against
its own templates (n_theta angles, M levels, a GEMM precision per size).
Every size is one sw_align_batch call; the calls of all sizes are captured
once, back to back on one stream, into a CUDA graph, and each later batch of
the same shapes is one graph launch: no per-kernel host work, no Python
between the sizes.

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
                 cache_path: str | None = None):
        import torch
        self.torch = torch
        self.device = device
        self.mode = mode
        self.al = swalign.Aligner(device)
        self.buckets = []
        for b in buckets:
            Nq, Nt = b.queries.shape[0], b.templates.shape[0]
            rows = Nq * Nt if mode == 0 else Nq
            if b.out is None:
                b.out = torch.empty((rows, 40), dtype=torch.uint8, device=b.queries.device)
            if autotune:
                self.al.autotune(b.params, cache_path)
            self.buckets.append(b)
        for b in self.buckets:  # the workspace grows to the largest size
            self.al.reserve(b.params, b.queries.shape[0], b.templates.shape[0])
        self.stream = torch.cuda.Stream(device=device)
        with torch.cuda.stream(self.stream):
            self._run_all()  # eager pass: one-time setup happens outside the capture
        self.stream.synchronize()
        self.launches_per_replay = -self.al.launch_count()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream, capture_error_mode="thread_local"):
            self._run_all()
        self.launches_per_replay += self.al.launch_count()

    def _run_all(self):
        for b in self.buckets:
            self.al.align_batch(b.queries, b.templates, b.params, mode=self.mode, out=b.out,
                                stream=self.torch.cuda.current_stream())

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
        self.al.profile(True)
        self.al.profile_read()
        try:
            with self.torch.cuda.stream(self.stream):
                for b in self.buckets:
                    self.al.align_batch(b.queries, b.templates, b.params, mode=self.mode,
                                        out=b.out, stream=self.stream)
                    out[b.L] = {k: v[0] for k, v in self.al.profile_read().items()}
        finally:
            self.al.profile(False)
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
        self.al.close()


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
