"""Benchmark: aligned image pairs per second on the many-to-many workload.

Workload (one step): 4096 query images against 256 templates, 128 x 128
cells, n = 256 angles, M = 128 quantile levels -- every pair aligned over all
256 rotations with the closed-form translation, through the C ABI call
sw_align_batch.  Projections by the paper's Fourier-slice (NUFFT) projector
(B = 192 bins); the linear-splat projector is reported as a variant.  Synthetic, seeded inputs (rotated / shifted / warped copies of
Gaussian-blob templates).  The device number times K steps with inputs
resident in HBM; "e2e" times the same call with the inputs copied from pinned
host memory and the results copied back inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|bf16|fp16]
  python bench.py --impl reference ...   (the FP64 CPU oracle, bounded sample)
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "aligned image pairs/s (128x128, 256 angles) FP32 vs BF16; p99 request latency"
PROJECTOR_NAMES = {"slice": "Fourier slice: type-2 NUFFT of the cell image, band-limited rows "
                            "(Sec. 2.3)",
                   "splat": "pixel-driven linear splat"}
NQ, NT, L, N_THETA, M_LEVELS = 4096, 256, 128, 256, 128
FP32_LANES, SM_MAX_MHZ_NOMINAL = 128, 2070.0   # FP32 lanes per SM; nominal max SM clock
B_BINS = 2 * math.ceil((L - 1) / math.sqrt(2.0)) + 2   # default bin count at L = 128
WORKLOAD = f"many-to-many {NQ}x{NT} pairs, {L}x{L}, n={N_THETA}, M={M_LEVELS}"
# algorithmic work per unit of the projection (the roofline counts only these flops)
PROJ_FLOPS_PER_CELL_ANGLE = 8           # s = <x, e> (FMA), frac, 1-t, two FMA accumulations
SLICE_W = 9                              # spreading kernel taps per axis


def slice_bins(Lc):
    """Bins (= oversampled grid) of the Fourier-slice projector at side Lc."""
    B0 = 2 * math.ceil((Lc - 1) / math.sqrt(2.0)) + 2
    need = max(B0, (3 * Lc + 1) // 2)
    return 32 * ((need + 31) // 32)


def slice_flops_per_image(Lc, n, B):
    """Transform arithmetic of the slice projector per image: complex FFTs of
    length B counted 5 B log2 B (ceil(L/2) column pairs, B/2 + W kept grid
    rows, n/4 inverse transforms of two angles) and 4 flops per tap of the
    W x W interpolation at each of the (n/2)(B/2 + 1) slice samples."""
    fft = 5.0 * B * math.log2(B)
    return ((Lc + 1) // 2 + B // 2 + SLICE_W + n // 4) * fft + \
        (n // 2) * (B // 2 + 1) * SLICE_W * SLICE_W * 4.0


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per 128 x 128 image
# of the slice projector kernel, from one ncu capture of a 512-image launch
# (33,824,768 + 40,143,104 bytes); None once that kernel changes.
SLICE_DRAM_BYTES_PER_IMAGE = 73967872 / 512
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per 128 x 128 image
# of the four-angle projection kernel, from one ncu capture of its 2112-image
# launch (2048 queries and 64 templates in one launch: 277,210,112 bytes);
# None once that kernel changes.
PROJ_DRAM_BYTES_PER_IMAGE = 277210112 / 2112
CORR_FLOPS_PER_PAIR_FREQ = 8 * M_LEVELS  # complex multiply-add per level


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16", "fp32_simt"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-uneven", action="store_true")
    ap.add_argument("--metric", default="sw2", choices=["sw2", "rfsw2", "msw2"],
                    help="distance of the main workload (profiling runs)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--projector", default="slice", choices=["splat", "slice"],
                    help="projection of the headline step: Fourier slice (default) or splat")
    ap.add_argument("--configs", action="store_true",
                    help="also time the single-pair, one-reference and random-dense "
                         "configurations (GPU and oracle) and print them as a second line")
    ap.add_argument("--partition", default="replicas", choices=["replicas", "rows"],
                    help="N > 1: independent replicas of the workload (weak scaling) or one "
                         "workload with its query rows split over the ranks (strong scaling)")
    ap.add_argument("--serve-requests", type=int, default=200)
    # 6 slots of at most 128 images: p99 3.2 / 3.6 ms (BF16 / FP32) against 3.9 / 4.1 ms with
    # 3 slots of 512 images, for 5% less saturation throughput (400 requests, one GB300)
    ap.add_argument("--serve-slots", type=int, default=6,
                    help="serving: concurrent slots (streams with their own context)")
    ap.add_argument("--serve-max-batch", type=int, default=128,
                    help="serving: most images per batch (larger requests are split)")
    ap.add_argument("--serve-only", action="store_true",
                    help="profiling runs only: print the serving block alone")
    ap.add_argument("--uneven-only", action="store_true",
                    help="profiling runs only: print the uneven-batch block alone")
    ap.add_argument("--nq", type=int, default=NQ, help="queries (profiling runs only)")
    ap.add_argument("--nt", type=int, default=NT, help="templates (profiling runs only)")
    ap.add_argument("--project-L", type=int, default=0,
                    help="profiling runs only: time the projection of 512 synthetic images of "
                         "this size and print one line")
    ap.add_argument("--project-n", type=int, default=256,
                    help="profiling runs only: angles of --project-L")
    ap.add_argument("--project-half", action="store_true",
                    help="profiling runs only: --project-L on images of side L/2 upsampled 2 x 2")
    return ap.parse_args()


def fp32_peak(device):
    """FP32 FMA peak of the device: measured by the library's FFMA probe
    (sw_measure_fp32_fma, at the clocks the GPU runs at), with the unit-count
    figure (SMs x 128 lanes x 2 x max SM clock) beside it."""
    import torch

    from paper_2503_13756_gb300 import swalign
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    peaks, _ = measured_peaks()
    nominal = sms * FP32_LANES * 2 * peaks.get("sm_max_mhz", SM_MAX_MHZ_NOMINAL) * 1e6 / 1e12
    tf, ms = swalign.measure_fp32_fma(device)
    return {"tflops": tf, "unit_count_tflops": nominal, "sms": sms, "probe_ms": ms,
            "source": "measured: FFMA probe (sw_measure_fp32_fma), best of 10 launches"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": SM_MAX_MHZ_NOMINAL}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        rows = []
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return None
        sm = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2])
                          if v.lower() in ("active", "1", "yes")})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


def rank_seed(rank: int) -> int:
    """Seed of rank r's images in the replica (weak-scaling) mode: every
    replica aligns its own workload, so no two ranks repeat each other's
    pairs."""
    from paper_2503_13756_gb300 import synth
    return synth.SEED_BASE + 2 + 1000 * rank


def row_block(nq: int, world: int, rank: int):
    """Query rows [lo, hi) of rank r in the row-partition (strong-scaling)
    mode: one fixed workload whose query rows are split as evenly as
    possible, the templates replicated on every rank.  Pairs are independent,
    so no rank needs another's data."""
    base, extra = divmod(nq, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("SW_BENCH_GLOO") is None else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def sample_size(projector):
    """Queries (and templates) of the oracle's sample: the first s x s pairs
    of the workload (the oracle's slice projector sums the slice samples
    directly, seconds per image, hence the smaller sample)."""
    return 32 if projector == "slice" else 160


def parity_of(gpu, ref, S, rel):
    """Measured error of the GPU results against the oracle's on the same
    pairs: plain relative error of d2 (no floor), absolute error in units of
    S = (N_i + N_j) / (n M), the ratio to the test bar rel max(d2, 0.1 S),
    rotation agreement and the largest shift error where the rotations agree."""
    g, r = gpu.reshape(-1), ref.reshape(-1)
    S = np.asarray(S, dtype=np.float64).reshape(-1)
    err = np.abs(g["d2"] - r["d2"])
    same = g["best_l"] == r["best_l"]
    dl = np.abs((g["best_l"] - r["best_l"] + N_THETA // 2) % N_THETA - N_THETA // 2)
    ds = np.abs(g["shift"] - r["shift"]).max(axis=1)
    relerr = err / r["d2"]
    return {"pairs": int(g.size), "argmin_same": float(same.mean()),
            "argmin_within_1_bin": float((dl <= 1).mean()),
            "max_rel_d2": float(relerr.max()), "median_rel_d2": float(np.median(relerr)),
            "frac_rel_d2_above_1e-5": float((relerr > 1e-5).mean()),
            "max_abs_d2_over_S": float((err / S).max()),
            "worst_ratio_to_bar": float((err / (rel * np.maximum(r["d2"], 0.1 * S) + 1e-12)).max()),
            "bar": f"{rel:g} max(d2, 0.1 S)",
            "max_shift_err": float(ds[same].max()) if same.any() else None,
            "min_d2_over_S": float((r["d2"] / S).min())}


def cpu_baseline(data, projector="slice", gpu=None, norms=None, s=None):
    """The FP64 oracle as it stands, on the host cores, on the first s x s
    pairs of the workload (sample_size), timed.  With `gpu` ({name: (block
    [s][s], source pairs [s])} of sw_result records from the timed runs) and
    `norms` (the GPU's centred quantile norms of the sample's queries, their
    templates and their source templates), the oracle's results on the same
    pairs -- the timed block, and each sampled query with its own template
    (well aligned: d2 / S ~ 1e-4) -- give the measured error per result."""
    import oracle
    if s is None:
        s = min(sample_size(projector), len(data["queries"]), len(data["templates"]))
    proj = int(projector == "slice")
    q = data["queries"][:s].astype(np.float64)
    t = data["templates"][:s].astype(np.float64)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    ref = oracle.align_all_pairs(q, t, N_THETA, M_LEVELS, nthreads=cores, projector=proj)
    dt = time.perf_counter() - t0
    pairs = s * s
    out = {"value": pairs / dt, "unit": "pairs/s", "cores": cores, "kind": "oracle",
           "sample": f"first {s} queries x {s} templates of the workload "
                     f"({pairs} pairs, {dt:.1f} s)"}
    parity = None
    if gpu:
        src = np.asarray(data["source"][:s])
        ts = data["templates"][src].astype(np.float64)
        ref_src = oracle.align_all_pairs(q, ts, N_THETA, M_LEVELS, nthreads=cores,
                                         projector=proj)[np.arange(s), np.arange(s)]
        nq_, nt_, ns_ = norms
        S_blk = (nq_[:, None] + nt_[None, :]) / (N_THETA * M_LEVELS)
        S_src = (nq_ + ns_) / (N_THETA * M_LEVELS)
        parity = {"oracle": "FP64 oracle from the same FP32 images (independent code)",
                  "block": f"first {s} queries x {s} templates ({pairs} pairs)",
                  "source_pairs": f"the first {s} queries with their own templates "
                                  "(well-aligned pairs)"}
        for name, (blk, srcp) in gpu.items():
            rel = 1e-2 if name in ("bf16", "fp16") else 1e-5
            parity[name] = {"block": parity_of(blk, ref, S_blk, rel),
                            "source_pairs": parity_of(srcp, ref_src, S_src, rel)}
    return out, parity


def serving_block(args, device):
    """Continuous-batching serving of Poisson requests against a 1000-template
    bank at 256 x 256 (n = 360, M = 256): latency percentiles and throughput."""
    from paper_2503_13756_gb300 import serving, swalign, synth
    bank = synth.serving_bank(n_templates=1000, L=256)
    pool = synth.serving_pool(bank, pool_size=256)
    sched = synth.serving_schedule(args.serve_requests, rate_hz=200.0, max_images=512, Lb=256)
    out = {"workload": "Poisson 200 req/s, 1-512 images per request (log-uniform), L=128 "
                       "(upsampled) or 256, bank of 1000 templates at 256x256, n=360, M=256, "
                       "best template per query",
           "projector": PROJECTOR_NAMES[args.projector],
           "requests": args.serve_requests, "slots": args.serve_slots,
           "max_batch_images": args.serve_max_batch}
    for prec in ("bf16", "fp32"):
        p = swalign.make_params(256, 360, 256, precision=prec, projector=args.projector)
        eng = serving.ServingEngine(bank["templates"], p, n_slots=args.serve_slots,
                                    max_batch_images=args.serve_max_batch,
                                    device=device, autotune=not args.no_autotune)
        try:
            warm = serving.make_requests(pool, synth.serving_schedule(8, 1000.0, 64, Lb=256))
            eng.run(warm, realtime=False)
            eng.batches, eng.batch_sizes = 0, []
            reqs = serving.make_requests(pool, sched)
            st = eng.run(reqs, realtime=True)
            hits = float(np.mean(np.concatenate(
                [r.results["template_index"].astype(int) == r.source for r in reqs])))
            st["source_template_found"] = hits
            # saturation: the same requests offered all at once (load above
            # capacity), so the slots never wait for arrivals; pairs/s is then
            # the engine's capacity and latency is mostly queueing
            eng.batches, eng.batch_sizes = 0, []
            sat = eng.run(serving.make_requests(pool, sched), realtime=False)
            st["saturation"] = {"pairs_per_s": sat["pairs_per_s"], "wall_s": sat["wall_s"],
                                "latency_ms": sat["latency_ms"], "batches": sat["batches"],
                                "mean_batch_images": sat["mean_batch_images"],
                                "offered": "all requests at t = 0"}
            out[prec] = st
        finally:
            eng.close()
    return out


def uneven_block(args, device):
    """Uneven batch: 20,000 queries with L in {64, 96, 128, 192, 256}
    (0.3/0.25/0.2/0.15/0.1), 64 templates per size, n = 256, M = L, BF16 GEMM,
    all sizes in one CUDA graph with autotuned launch shapes.  Device time per
    graph launch (CUDA events on the graph's stream), and the same calls made
    eagerly for comparison."""
    import torch

    import tempfile

    from paper_2503_13756_gb300 import synth, uneven
    batch = synth.uneven_batch()
    # one tuning cache for both graphs below: the same launch shapes in each
    tune_cache = os.path.join(tempfile.mkdtemp(prefix="swtune"), "tune.txt")
    g = uneven.UnevenGraph(uneven.buckets_from(batch, 256, "bf16", device,
                                               projector=args.projector), mode=0,
                           device=device, autotune=not args.no_autotune, cache_path=tune_cache)
    try:
        st = g.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(2):
            g.replay()
        st.synchronize()
        reps = 5
        e0.record(st)
        for _ in range(reps):
            g.replay()
        e1.record(st)
        e1.synchronize()
        ms_graph = e0.elapsed_time(e1) / reps
        e0.record(st)
        for _ in range(reps):
            g.run_eager()
        e1.record(st)
        e1.synchronize()
        ms_eager = e0.elapsed_time(e1) / reps
        res = g.results()
        ok = all(bool(np.all(r["status"] == 0)) for r in res.values())
        stages = {int(k): {s_: round(v, 4) for s_, v in d.items()}
                  for k, d in g.stage_times().items()}
        # the same sizes back to back on one stream (one branch), for comparison
        gs = uneven.UnevenGraph(g.buckets, mode=0, device=device, concurrent=False,
                                autotune=not args.no_autotune, cache_path=tune_cache)
        try:
            for _ in range(2):
                gs.replay()
            gs.stream.synchronize()
            e0.record(gs.stream)
            for _ in range(reps):
                gs.replay()
            e1.record(gs.stream)
            e1.synchronize()
            ms_seq = e0.elapsed_time(e1) / reps
            same = all(np.array_equal(gs.results()[L]["d2"], res[L]["d2"]) for L in res)
        finally:
            gs.close()
        return {"workload": "uneven 20,000 queries, L in {64,96,128,192,256}, 64 templates per L, "
                            "n=256, M=L, BF16 GEMM, one CUDA graph",
                "projector": PROJECTOR_NAMES[args.projector],
                "pairs": g.pairs, "ms_per_graph": ms_graph, "pairs_per_s": g.pairs / (ms_graph / 1e3),
                "graph": "one branch per size (own context and stream), forked and joined "
                         "inside the graph",
                "sequential_ms_per_graph": ms_seq, "sequential_results_identical": bool(same),
                "eager_ms": ms_eager, "kernels_per_graph": g.launches_per_replay,
                "queries_per_L": {int(b.L): int(b.queries.shape[0]) for b in g.buckets},
                "stages_ms_per_L": stages,
                "status_ok": ok}
    finally:
        g.close()
        del g, batch
        torch.cuda.empty_cache()


def configs_block(device, projector="slice"):
    """The other configurations of the method, each on the GPU (device time
    from CUDA events; single-pair latency also as host wall time) and the
    FP64 oracle on a bounded sample (1 thread and all host threads), with the
    given projector:
      single pair 64 x 64, n = 360, M = 128, all rotations + translation;
      one reference x 10,000 queries, 128 x 128, n = 512, M = 256;
      random dense U[0,1) images, L = n = M in {32, 64, 96, 128}, rotation only
      (the paper's Table 3 timing setting), one pair per call and batched."""
    import torch

    import oracle
    from paper_2503_13756_gb300 import swalign, synth
    al = swalign.Aligner(device)
    out = {"projector": PROJECTOR_NAMES[projector]}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cores = os.cpu_count() or 1

    def dev_ms(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    def wall_ms(fn, reps):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(1e3 * (time.perf_counter() - t0))
        return float(np.median(ts))

    proj = int(projector == "slice")

    def oracle_rate(q, t, n, M, translation, threads):
        t0 = time.perf_counter()
        oracle.align_all_pairs(q, t, n, M, translation=translation, nthreads=threads,
                               projector=proj)
        return len(q) * len(t) / (time.perf_counter() - t0)

    # ---- single pair
    d = synth.single_pair()
    f, g = d["f"].astype(np.float32), d["g"].astype(np.float32)
    p = swalign.make_params(64, 360, 128, projector=projector)
    fd, gd = torch.from_numpy(f).cuda(device), torch.from_numpy(g).cuda(device)
    al.reserve(p, 1, 1)
    fn = lambda: al.align_all_rotations(fd, gd, p)
    out["single_pair_64_n360_M128"] = {
        "device_ms": dev_ms(fn, 50), "host_wall_ms": wall_ms(fn, 50),
        "oracle_pairs_per_s_1thread": oracle_rate(f[None].astype(np.float64),
                                                  g[None].astype(np.float64), 360, 128, 1, 1)}
    # ---- one reference x 10,000 queries
    d = synth.one_reference_batch()
    q, ref = d["queries"], d["reference"]
    p = swalign.make_params(128, 512, 256, projector=projector)
    qd, rd = torch.from_numpy(q).cuda(device), torch.from_numpy(ref).cuda(device)
    res = torch.empty((len(q), 40), dtype=torch.uint8, device=qd.device)
    al.autotune(p)
    al.reserve(p, len(q), 1)
    ms = dev_ms(lambda: al.align_batch(qd, rd, p, out=res), 5)
    nsub = 64 if proj else 256  # the oracle's slice sums take seconds per image
    sub = q[:nsub].astype(np.float64)
    out["one_reference_10000_n512_M256"] = {
        "pairs_per_s": len(q) / (ms / 1e3), "ms_per_batch": ms,
        "oracle_pairs_per_s": oracle_rate(sub, ref.astype(np.float64), 512, 256, 1, cores),
        "oracle_threads": cores, "oracle_sample": f"first {nsub} queries"}
    del qd, res
    # ---- random dense, rotation only, L = n = M
    wa = {}
    for Lw in (32, 64, 96, 128):
        x = synth.random_dense(Lw, count=1024 + 64, seed=synth.SEED_BASE + 9 + Lw)
        p = swalign.make_params(Lw, Lw, Lw, translation=0, projector=projector)
        xd = torch.from_numpy(x).cuda(device)
        one = lambda: al.align_all_rotations(xd[0], xd[1], p)
        res = torch.empty((1024 * 64, 40), dtype=torch.uint8, device=xd.device)
        al.reserve(p, 1024, 64)
        ms_b = dev_ms(lambda: al.align_batch(xd[:1024], xd[1024:], p, out=res), 5)
        xs = x[:32].astype(np.float64)
        wa[str(Lw)] = {"single_pair_host_wall_ms": wall_ms(one, 30),
                       "single_pair_device_ms": dev_ms(one, 30),
                       "batched_pairs_per_s": 1024 * 64 / (ms_b / 1e3),
                       "oracle_pairs_per_s_1thread": oracle_rate(xs[:4], xs[4:8], Lw, Lw, 0, 1),
                       "paper_pairs_per_s_skylake": {32: 769, 64: 370, 96: 159, 128: 103}[Lw]}
        del xd, res
    out["random_dense_rotation_only"] = wa
    # ---- max-sliced W2 over rotations: 512 x 64 pairs of the many-to-many images
    d = synth.many_to_many(n_queries=512, n_templates=64)
    qd = torch.from_numpy(d["queries"]).cuda(device)
    td = torch.from_numpy(d["templates"]).cuda(device)
    p = swalign.make_params(128, 256, 128, metric="msw2", projector=projector)
    res = torch.empty((512 * 64, 40), dtype=torch.uint8, device=qd.device)
    al.reserve(p, 512, 64)
    al.profile(True)
    al.profile_read()
    ms = dev_ms(lambda: al.align_batch(qd, td, p, out=res), 3)
    st_m = al.profile_read()
    al.profile(False)
    k_ms = st_m.get("decide", (0.0, 1))[0] / st_m.get("decide", (0.0, 1))[1]
    flops = 512 * 64 * 256 * 256 * 128 * 3  # subtract + fused multiply-add per term
    fp = fp32_peak(device)
    peak = fp["tflops"]
    out["max_sliced_512x64_n256_M128"] = {
        "pairs_per_s": 512 * 64 / (ms / 1e3), "ms_per_batch": ms,
        "k_msw": {"ms": k_ms, "achieved_tflops": flops / (k_ms / 1e3) / 1e12, "peak": peak,
                  "frac": flops / (k_ms / 1e3) / 1e12 / peak,
                  "peak_source": fp["source"], "unit_count_peak": fp["unit_count_tflops"]}}
    al.close()
    torch.cuda.empty_cache()
    return out


def run_reference(args, world, rank):
    """Reference arm: the FP64 CPU oracle on a bounded sample per step: 16
    queries x 16 templates of the workload's images (their transforms and
    256 pair searches; about 2 s on 16 cores), a different block each step."""
    if rank != 0:
        return
    from paper_2503_13756_gb300 import synth
    import oracle
    oracle.build()
    data = synth.many_to_many(n_queries=64, n_templates=64)
    slice_proj = args.projector == "slice"
    sq = st = 16
    cores = os.cpu_count() or 1
    times = []
    for k in range(args.warmup + args.steps):
        i0 = (k * sq) % (64 - sq)
        q = data["queries"][i0:i0 + sq].astype(np.float64)
        t = data["templates"][i0:i0 + st].astype(np.float64)
        t0 = time.perf_counter()
        oracle.align_all_pairs(q, t, N_THETA, M_LEVELS, nthreads=cores,
                               projector=int(slice_proj))
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    value = sq * st / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "Nq": NQ, "Nt": NT, "L": L, "n_theta": N_THETA,
                   "n_levels": M_LEVELS, "projector": PROJECTOR_NAMES[args.projector],
                   "step_sample": f"{sq}x{st} pairs per step"},
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sq} queries x {st} templates per step, {args.steps} steps"},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def project_only(args):
    """Profiling aid: the projector alone on 512 blob-mixture images of side
    --project-L (n = --project-n, M = 128), 2 warm-up and 5 timed calls.
    With --project-half the images are summed 2 x 2 to side L/2 and projected
    as their 2 x 2 upsampled L x L images (sw_project_upsampled)."""
    import torch

    from paper_2503_13756_gb300 import swalign, synth
    Lp = args.project_L
    al = swalign.Aligner(0)
    rng = np.random.default_rng(synth.SEED_BASE + 7)
    imgs = np.ascontiguousarray(synth.render(synth.draw_mixtures(rng, 512, Lp, ncomp=(2, 4)), Lp),
                                dtype=np.float32)
    if args.project_half:
        imgs = np.ascontiguousarray(
            imgs.reshape(512, Lp // 2, 2, Lp // 2, 2).sum(axis=(2, 4)), dtype=np.float32)
    pa = swalign.make_params(Lp, args.project_n, M_LEVELS, projector=args.projector)
    x = torch.from_numpy(imgs).cuda()
    run = al.project_upsampled if args.project_half else al.project
    for _ in range(2):
        run(x, pa)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        run(x, pa)
    e1.record()
    e1.synchronize()
    us = e0.elapsed_time(e1) / 5 / 512 * 1e3
    print(json.dumps({"profile": "projection only", "L": Lp, "n": args.project_n,
                      "half_size": bool(args.project_half), "projector": args.projector,
                      "images": 512, "us_per_image": us}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        # rank 0 alone times the oracle; no collective, so no process group
        run_reference(args, int(os.environ.get("WORLD_SIZE", "1")),
                      int(os.environ.get("RANK", "0")))
        return
    world, rank, local = dist_setup()
    if args.project_L:
        project_only(args)
        return
    if args.serve_only:
        print(json.dumps({"serving": serving_block(args, local)}), flush=True)
        return
    if args.uneven_only:
        print(json.dumps({"uneven": uneven_block(args, local)}), flush=True)
        return
    import torch

    from paper_2503_13756_gb300 import swalign, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nq_all, nt = args.nq, args.nt
    if args.partition == "rows":
        # one workload on every rank; this rank aligns its block of query rows
        data = synth.many_to_many(n_queries=nq_all, n_templates=nt, seed=rank_seed(0))
        lo, hi = row_block(nq_all, world, rank)
        data = dict(data, queries=data["queries"][lo:hi], source=data["source"][lo:hi])
    else:
        data = synth.many_to_many(n_queries=nq_all, n_templates=nt, seed=rank_seed(rank))
    nq = len(data["queries"])
    pairs_per_rank = nq * nt
    al = swalign.Aligner(local)
    p = swalign.make_params(L, N_THETA, M_LEVELS, precision=args.precision, metric=args.metric,
                            projector=args.projector)
    q_h = torch.from_numpy(data["queries"]).pin_memory()
    t_h = torch.from_numpy(data["templates"]).pin_memory()
    q_d, t_d = q_h.to(dev), t_h.to(dev)
    out = torch.empty((nq * nt, 40), dtype=torch.uint8, device=dev)
    tune = None if args.no_autotune else list(al.autotune(p))
    al.reserve(p, nq, nt)
    stream = torch.cuda.current_stream()
    fp32pk = fp32_peak(local)
    # results of the oracle's sample (the first s x s pairs and the first s
    # queries with their own templates), kept from every run of the sample's
    # projector and distance for the measured error per result
    s_par = min(sample_size(args.projector), nq, nt)
    src_idx = torch.as_tensor(np.asarray(data["source"][:s_par]), device=dev)
    gpu_sample = {}

    def keep_sample(name):
        o3 = out.view(nq, nt, 40)
        gpu_sample[name] = (
            swalign.results_to_numpy(o3[:s_par, :s_par].contiguous()).reshape(s_par, s_par),
            swalign.results_to_numpy(o3[torch.arange(s_par, device=dev), src_idx].contiguous()))

    for _ in range(max(3, args.warmup)):
        al.align_batch(q_d, t_d, p, out=out)
    torch.cuda.synchronize()
    barrier(world)

    # ---- device-timed steps (inputs resident), kernel events on the same stream
    al.profile(True)
    al.profile_read()
    n0 = al.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            al.align_batch(q_d, t_d, p, out=out)
        e1.record(stream)
        e1.synchronize()
    launches = al.launch_count() - n0
    stages = al.profile_read()
    al.profile(False)
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = max_over_ranks(ms, world, dev)
    total_pairs = sum_over_ranks(pairs_per_rank, world, dev)
    value = total_pairs / (ms_max / 1e3)
    res = swalign.results_to_numpy(out[:nt])
    assert np.all(res["status"] == 0)
    if args.metric == "sw2":
        keep_sample(args.precision)

    # ---- end to end: pinned host inputs -> device -> results back, per step.
    # Every step copies its inputs in and its results out inside the timed
    # region; two buffer sets let step k+1's upload and step k-1's download run
    # on copy streams while step k computes (the order a serving loop uses).
    # Measured right after the device-resident steps, before the variants
    # heat the GPU, with its own clock samples.
    e2e = None
    if not args.no_e2e:
        cs_in, cs_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
        qb = [q_d, torch.empty_like(q_d)]
        tb = [t_d, torch.empty_like(t_d)]
        ob = [out, torch.empty_like(out)]
        oh = [torch.empty((nq * nt, 40), dtype=torch.uint8).pin_memory() for _ in range(2)]
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_comp = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]

        def pipeline(nsteps, spans=None):
            # spans: optional list that receives, per step, timing events around
            # the upload, the compute and the download as they ran in the pipeline
            for k in range(nsteps):
                b = k % 2
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)] if spans is not None else None
                with torch.cuda.stream(cs_in):
                    if k >= 2:
                        cs_in.wait_event(ev_comp[b])  # step k-2 has read these inputs
                    if ev: ev[0].record(cs_in)
                    qb[b].copy_(q_h, non_blocking=True)
                    tb[b].copy_(t_h, non_blocking=True)
                    ev_in[b].record(cs_in)
                    if ev: ev[1].record(cs_in)
                stream.wait_event(ev_in[b])
                if k >= 2:
                    stream.wait_event(ev_out[b])      # step k-2's results are out
                if ev: ev[2].record(stream)
                al.align_batch(qb[b], tb[b], p, out=ob[b], stream=stream)
                ev_comp[b].record(stream)
                if ev: ev[3].record(stream)
                with torch.cuda.stream(cs_out):
                    cs_out.wait_event(ev_comp[b])
                    if ev: ev[4].record(cs_out)
                    oh[b].copy_(ob[b], non_blocking=True)
                    ev_out[b].record(cs_out)
                    if ev: ev[5].record(cs_out)
                if ev: spans.append(ev)
            return ev_out[(nsteps - 1) % 2]

        pipeline(2)
        torch.cuda.synchronize()
        # the host link's rate on this machine: one upload of a step's inputs and
        # one download of its results alone (the pipeline hides them behind
        # the compute only while they take less than a step)
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(cs_in):
            h0.record(cs_in)
            for _ in range(3):
                qb[1].copy_(q_h, non_blocking=True)
                tb[1].copy_(t_h, non_blocking=True)
            h1.record(cs_in)
        h1.synchronize()
        h2d_ms = h0.elapsed_time(h1) / 3
        with torch.cuda.stream(cs_out):
            h0.record(cs_out)
            for _ in range(3):
                oh[1].copy_(ob[1], non_blocking=True)
            h1.record(cs_out)
        h1.synchronize()
        d2h_ms = h0.elapsed_time(h1) / 3
        torch.cuda.synchronize()
        barrier(world)
        with ClockSampler(local) as clk_e2e:
            torch.cuda.synchronize()
            e0.record(stream)
            cs_in.wait_stream(stream)
            last = pipeline(args.steps)
            cs_out.wait_event(last)
            e1.record(cs_out)
            e1.synchronize()
        torch.cuda.synchronize()
        assert torch.equal(oh[(args.steps - 1) % 2], ob[(args.steps - 1) % 2].cpu())
        ms_e2e = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
        # one more pass of the same pipeline, outside the timed region, with
        # events around each copy and each compute: how long they took while
        # overlapped (a copy that slows under the compute, or a compute that
        # slows under the copies, shows here)
        spans = []
        pipeline(args.steps, spans)
        torch.cuda.synchronize()
        med = lambda xs: float(np.median(xs))
        in_pipe = {"h2d_ms": med([e[0].elapsed_time(e[1]) for e in spans]),
                   "compute_ms": med([e[2].elapsed_time(e[3]) for e in spans]),
                   "d2h_ms": med([e[4].elapsed_time(e[5]) for e in spans]),
                   "step_ms": med([a[3].elapsed_time(b[3]) for a, b in zip(spans, spans[1:])])}
        e2e = {"value": total_pairs / (ms_e2e / 1e3), "unit": "pairs/s",
               "h2d_bytes_per_step": int(q_h.numel() * 4 + t_h.numel() * 4),
               "d2h_bytes_per_step": int(oh[0].numel()),
               "pipeline": "inputs of step k+1 uploaded and results of step k-1 read back "
                           "on copy streams while step k computes (two buffer sets)",
               "h2d_ms_alone": h2d_ms, "d2h_ms_alone": d2h_ms,
               "h2d_gbs_alone": (q_h.numel() + t_h.numel()) * 4 / (h2d_ms / 1e3) / 1e9,
               "in_pipeline_median": in_pipe,
               "clocks": clk_e2e.summary()}

    # ---- the same workload with the tensor-core correlation (BF16 / FP16)
    variants = {}
    if args.precision == "fp32" and args.metric == "sw2" and not args.no_variants:
        other = "splat" if args.projector == "slice" else "slice"
        for name in ("bf16", "fp16", "fp32_simt", "rfsw2_fp32", "rfsw2_bf16", other + "_fp32"):
            metric = "rfsw2" if name.startswith("rfsw2") else "sw2"
            prec = name.split("_", 1)[1] if "_" in name and not name.startswith("fp32") else name
            proj = other if name.startswith(other) else args.projector
            pv = swalign.make_params(L, N_THETA, M_LEVELS, precision=prec, metric=metric,
                                     projector=proj)
            if not args.no_autotune:
                al.autotune(pv)
            al.reserve(pv, nq, nt)
            for _ in range(3):
                al.align_batch(q_d, t_d, pv, out=out)
            torch.cuda.synchronize()
            al.profile(True)
            al.profile_read()
            e0.record(stream)
            for _ in range(args.steps):
                al.align_batch(q_d, t_d, pv, out=out)
            e1.record(stream)
            e1.synchronize()
            st_v = al.profile_read()
            al.profile(False)
            ms_v = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
            rv = swalign.results_to_numpy(out[:nt])
            if metric == "sw2" and proj == args.projector:
                keep_sample(prec)
            corr_ms = st_v.get("corr", (0.0, 1))[0] / args.steps
            # the ramp-filtered metric correlates both parts: K = 4M instead of 2M
            flops = (nq * nt * (N_THETA // 2) * CORR_FLOPS_PER_PAIR_FREQ
                     * (2 if metric == "rfsw2" else 1))
            peaks_v, _ = measured_peaks()
            tf = flops / (corr_ms / 1e3) / 1e12 if corr_ms > 0 else None
            simt = prec == "fp32_simt"
            peak_v = fp32pk["tflops"] if simt else peaks_v.get("bf16_tflops")
            variants[name] = {
                "metric": {"sw2": "sliced W2", "rfsw2": "ramp-filtered sliced W2"}[metric],
                "projector": PROJECTOR_NAMES[proj],
                "value": sum_over_ranks(nq * nt, world, dev) / (ms_v / 1e3), "unit": "pairs/s",
                "ms_per_step": ms_v, "status_ok": bool(np.all(rv["status"] == 0)),
                "stages": {k: v[0] / args.steps for k, v in st_v.items()},
                "corr": {"achieved": tf, "unit": "TFLOP/s", "peak": peak_v,
                         "peak_kind": ("FP32 FMA, measured by the FFMA probe" if simt
                                       else "measured BF16 burst"),
                         "frac": tf / peak_v if tf else None,
                         "algorithmic_flops_per_launch": flops},
            }
        al.reserve(p, nq, nt)

    if rank != 0:
        return
    # ---- roofline of the dominant kernel
    peaks, peak_src = measured_peaks()
    nimg = nq + nt
    per_stage = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
                 for k, v in stages.items()}
    dom = max(stages, key=lambda k: stages[k][0])
    alu_peak = fp32pk["tflops"]
    alu_src = (f"{fp32pk['source']}; unit counts: {fp32pk['sms']} SMs x 128 FP32 lanes x 2 x "
               f"max SM clock = {fp32pk['unit_count_tflops']:.1f} TFLOP/s")
    if dom == "project" and args.projector == "slice":
        Bs = slice_bins(L)
        flops = args.steps * nimg * slice_flops_per_image(L, N_THETA, Bs)
        achieved = flops / (stages[dom][0] / 1e3) / 1e12
        per_launch = nimg / max(1.0, stages[dom][1] / args.steps)
        traffic = (SLICE_DRAM_BYTES_PER_IMAGE * per_launch
                   if SLICE_DRAM_BYTES_PER_IMAGE is not None else None)
        roof = {"kernel": "k_project_slice", "bound": "alu", "achieved": achieved,
                "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak,
                "traffic": traffic,
                "traffic_unit": "bytes per launch (average launch of the step)",
                "algorithmic_flops_per_image": slice_flops_per_image(L, N_THETA, Bs),
                "algorithmic_bytes_per_launch": per_launch * (L * L * 4 + (N_THETA // 2) * Bs * 4),
                "peak_source": alu_src,
                "binding_unit": "shared-memory pipe (tap loads) and instruction issue"}
        # the binding unit: tap loads (8-byte complex, W x W per slice sample)
        # against the shared-memory bandwidth (128 B per clock per SM)
        tap_bytes = (N_THETA // 2) * (Bs // 2 + 1) * SLICE_W * SLICE_W * 8
        smem_peak = fp32pk["sms"] * 128 * peaks.get("sm_max_mhz", SM_MAX_MHZ_NOMINAL) * 1e6 / 1e12
        smem_ach = args.steps * nimg * tap_bytes / (stages[dom][0] / 1e3) / 1e12
        roof["shared_memory"] = {
            "achieved": smem_ach, "peak": smem_peak, "unit": "TB/s", "frac": smem_ach / smem_peak,
            "tap_bytes_per_image": tap_bytes,
            "note": "tap loads only; the FFT exchanges and stores add the rest of the pipe's "
                    "load (ncu: L1/shared 89% of peak)"}
    elif dom == "project":
        flops = args.steps * nimg * L * L * (N_THETA // 2) * PROJ_FLOPS_PER_CELL_ANGLE
        achieved = flops / (stages[dom][0] / 1e3) / 1e12
        per_launch = nimg / max(1.0, stages[dom][1] / args.steps)
        traffic = (PROJ_DRAM_BYTES_PER_IMAGE * per_launch
                   if PROJ_DRAM_BYTES_PER_IMAGE is not None else None)
        roof = {"kernel": "k_project4", "bound": "alu", "achieved": achieved, "peak": alu_peak,
                "unit": "TFLOP/s", "frac": achieved / alu_peak, "traffic": traffic,
                "traffic_unit": "bytes per launch (average launch of the step)",
                "algorithmic_bytes_per_launch": per_launch * (L * L * 4 + (N_THETA // 2) * B_BINS * 4),
                "peak_source": alu_src}
    elif dom == "corr" and args.precision == "fp32_simt":
        flops = args.steps * nq * nt * (N_THETA // 2) * CORR_FLOPS_PER_PAIR_FREQ
        achieved = flops / (stages[dom][0] / 1e3) / 1e12
        roof = {"kernel": "k_corr_simt", "bound": "alu", "achieved": achieved, "peak": alu_peak,
                "unit": "TFLOP/s", "frac": achieved / alu_peak, "traffic": None,
                "peak_source": alu_src}
    else:
        roof = {"kernel": dom, "bound": "unknown", "achieved": None, "peak": None,
                "unit": None, "frac": None, "traffic": None}
    cpu, parity = None, None
    if not (args.no_cpu_baseline or world > 1):
        pn = swalign.make_params(L, N_THETA, M_LEVELS, projector=args.projector)
        norm = [al.quantiles(al.project(x, pn), pn)[2].cpu().numpy() for x in
                (q_d[:s_par], t_d[:s_par], t_d[src_idx])]
        cpu, parity = cpu_baseline(data, args.projector, gpu_sample, norm, s_par)
    serve = None if (args.no_serving or world > 1) else serving_block(args, local)
    unev = None if (args.no_uneven or world > 1) else uneven_block(args, local)
    line = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True,
        "scaling": "strong" if args.partition == "rows" else "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision.startswith("fp32") else args.precision,
        "data": "synthetic",
        "config": {"workload": WORKLOAD if (nq_all, nt) == (NQ, NT) else
                   f"many-to-many {nq_all}x{nt} pairs, {L}x{L}, n={N_THETA}, M={M_LEVELS}",
                   "Nq": nq_all, "Nq_per_rank": nq, "Nt": nt, "L": L, "n_theta": N_THETA,
                   "n_levels": M_LEVELS, "precision": args.precision, "translation": 1,
                   "projector": PROJECTOR_NAMES[args.projector],
                   "n_bins": swalign.bins_of(p),
                   "distance": {"sw2": "sliced W2", "rfsw2": "ramp-filtered sliced W2",
                                "msw2": "max-sliced W2"}[args.metric],
                   "correlation": ("none: every column pair, FP32 on the CUDA cores"
                                   if args.metric == "msw2" else
                                   {"fp32": "tcgen05, 3-term FP16 split, FP32 accumulate",
                                    "bf16": "tcgen05 BF16", "fp16": "tcgen05 FP16",
                                    "fp32_simt": "CUDA-core FP32"}[args.precision]),
                   "parallelism": (f"query rows of one {nq_all}x{nt} workload split over {world} "
                                   "ranks, templates replicated (strong)"
                                   if args.partition == "rows" else
                                   f"{world} independent replicas (weak)"),
                   "launch_shapes": tune,
                   "l2": "no flush: inputs (285 MB) and per-step workspace (>2 GB) exceed L2"},
        "roofline": roof, "peaks": peak_src, "fp32_peak": fp32pk, "stages": per_stage,
        "cpu_baseline": cpu, "parity": parity,
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clk.summary(),
        "variants": variants, "serving": serve, "uneven": unev,
    }
    print(json.dumps(line), flush=True)
    if args.configs and world == 1:
        print(json.dumps({"configs": configs_block(local, args.projector)}), flush=True)


if __name__ == "__main__":
    main()
