#!/usr/bin/env python
"""Throughput of the Barnes-Hut smooth distance + gradient (queries/s).

Workload: level-6 icosphere (81,920 triangles, radial noise 0.01), 262,144
queries (70 % in the shell |r-1| < 0.1, 30 % uniform in [-2,2]^3),
alpha = 200, beta = 0.5, leaf size 1, paper weights, fp32. One step is the
whole path: sd_build (validation, valences, Morton codes, radix sort, radix
tree, aggregates, gather), sd_query_order and sd_query (traversal with the
fused value + gradient) over one batch resident in HBM. The L2 is flushed
(a 256 MiB write) before every timed step; the flush is outside the step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Roofline: the traversal is bound by the FP32 pipe with the MUFU pipe as a
co-bound (its HBM traffic is a few MB per launch). Its work per launch is
the method's per-unit cost (METHOD_FLOPS, METHOD_MUFU) times the kernel's
work counts (Barnes-Hut tests, far-field accepts, exact leaf terms); the
peaks are measured on the GPU by the library's own FMA and ex2 probes,
scaled to the clock sampled during the timed region. The same figures are
reported for the nine (alpha, beta) cells of the icosphere workload and for
the street point queries (`cells`).

N > 1 runs under torchrun, one rank per GPU: every rank builds the same tree
and evaluates its own 262,144 queries (weak scaling, no data-path
collective); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "smooth-distance+grad queries/sec (BH)"
UNIT = "queries/s"
ALPHA, BETA, LEAF = 200.0, 0.5, 1
M_QUERIES = 262144

# Work of the method per unit, a hand count of the method's own arithmetic
# (not of any kernel): FP32 flops (add/sub/mul/min/max 1, FMA 2) and MUFU
# operations (exponential, (reciprocal) square root, reciprocal).
#   test   one Barnes-Hut test: point-to-AABB squared distance, one compare
#   far    an accepted far field: its distance, weight, exponential, LSE update
#   point / seg / tri   one exact leaf term: closest point, weight and its
#          gradient, LSE update
METHOD_FLOPS = {"test": 20, "far": 12, "point": 14, "seg": 45, "tri": 160}
METHOD_MUFU = {"test": 0, "far": 3, "point": 2, "seg": 3, "tri": 3}
# The traversal kernel's own hand count of the same units (its source:
# packed two-child test, branch-free far field, nested-Horner weight),
# reported beside the method's figure only.
KERNEL_FLOPS = {"test": 26, "far": 26, "tri": 362}
# tensor-core flops per query of the surrogate network, value and input
# gradient: forward 80x128 + 2 x 128x128 MACs (layer 1 padded to 80 inputs),
# backward 2 x 128x128 + 128x80 MACs, 2 flops per MAC
MLP_FLOPS = 2 * 2 * (80 * 128 + 2 * 128 * 128)
# the nine (alpha, beta) cells of the icosphere workload
CELL_ALPHAS = (50.0, 200.0, 1000.0)
CELL_BETAS = (0.25, 0.5, 1.0)


_SCENE = {}


def _street():
    """The street workload, generated once per process."""
    if "street" not in _SCENE:
        _SCENE["street"] = synth.config3_scene()
    return _SCENE["street"]


def _args():
    return _args_from(None)


def _args_from(argv):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--alpha", type=float, default=ALPHA)
    p.add_argument("--beta", type=float, default=BETA)
    p.add_argument("--leaf-size", type=int, default=LEAF)
    p.add_argument("--queries", type=int, default=M_QUERIES)
    p.add_argument("--no-extras", action="store_true", help="skip plain/e2e/cpu baseline and application legs")
    p.add_argument("--no-cells", action="store_true", help="skip the per-(alpha, beta) cell table")
    return p.parse_args(argv)


def _workload(args, rank=0):
    c = synth.config2(seed=1, m=args.queries)
    if rank:
        c["queries"] = synth.shell_queries(args.queries, 0.7, 0.9, 1.1, 2.0, seed=101 + rank)
    return c


def _config(args, n):
    return {"workload": f"icosphere-L6 81920 tris, {args.queries} queries/GPU (70% shell, 30% box), "
                        f"alpha={args.alpha:g}, beta={args.beta:g}, leaf={args.leaf_size}",
            "triangles": 81920, "queries_per_gpu": args.queries, "alpha": args.alpha, "beta": args.beta,
            "leaf_size": args.leaf_size,
            "step": "sd_build + sd_query_order (second stream, from the scene box on) + sd_query (value+grad)",
            "l2": "flushed (256 MiB write) before each timed step", "parallelism": f"replicated tree, dp{n}"}


def _src_hash():
    h = hashlib.sha256()
    for f in ("sd_query.cu", "sd_common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2108_10480_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _tensor_roofline(tflops):
    """The surrogate network's GEMM rate against the measured dense bf16
    peak of this machine's GPUs (burst: the kernel is timed alone), else the
    fallback figure."""
    peak, src = 1900.0, "fallback 1.9 PFLOP/s bf16"
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        if float(d.get("bf16_tflops", 0)) > 0:
            peak, src = float(d["bf16_tflops"]), "measured bf16 burst (cuBLAS)"
    except (OSError, ValueError, TypeError):
        pass
    return {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
            "peak_source": src}


def _traffic(kernel_hash):
    """Per-launch DRAM bytes of the traversal kernel from the committed ncu
    summary, or None if the kernel changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "k_traverse_ico6_traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    if d.get("src_hash") != kernel_hash:
        return None
    return d.get("dram_bytes_per_launch")


def _pipe_peaks(dev, clocks=None, target_ms=25.0):
    """FP32 and MUFU pipe rates measured on this GPU with the library's own
    probes (sd_peak_probe): fma.rn.f32 chains, fma.rn.f32x2 chains and
    ex2.approx chains on a full-occupancy grid (8 blocks of 256 threads per
    SM), each launch sized to about target_ms and timed with CUDA events
    (median of 5 after one warm-up). The FP32 peak is the better of the two
    FMA forms (an FMA is 2 flops); the MUFU peak is the ex2 rate."""
    import ctypes

    import torch

    from paper_2108_10480_gb300 import _native, lib
    L = lib()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = sms * 8
    sink = torch.empty(blocks * 256, device=dev)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ops = ctypes.c_double()
    rates = {}

    def launch(kind, iters):
        _native.check(L.sd_peak_probe(kind, blocks, iters, ctypes.c_void_p(sink.data_ptr()), ctypes.byref(ops),
                                      ctypes.c_void_p(stream.cuda_stream)), "sd_peak_probe")

    if clocks:
        clocks.begin("pipe_probes")
    for kind, name in ((0, "ffma"), (1, "ffma2"), (2, "ex2")):
        iters = 64
        launch(kind, iters)
        e0.record(stream)
        launch(kind, iters)
        e1.record(stream)
        torch.cuda.synchronize()
        iters = max(64, int(iters * target_ms / max(e0.elapsed_time(e1), 1e-3)))
        launch(kind, iters)
        ts = []
        for _ in range(5):
            e0.record(stream)
            launch(kind, iters)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        rates[name] = {"ops_per_s": ops.value / (statistics.median(ts) / 1e3), "ms": statistics.median(ts),
                       "iters": iters}
    if clocks:
        clocks.end("pipe_probes")
    fp32 = 2.0 * max(rates["ffma"]["ops_per_s"], rates["ffma2"]["ops_per_s"]) / 1e12
    return {"fp32_tflops": fp32, "mufu_gops": rates["ex2"]["ops_per_s"] / 1e9, "sms": sms, "blocks": blocks,
            "probes": {k: dict(v, ops_per_s=v["ops_per_s"]) for k, v in rates.items()},
            "source": "measured: sd_peak_probe fma.rn.f32 / fma.rn.f32x2 / ex2.approx.ftz.f32 chains, "
                      f"{blocks} x 256 threads, CUDA events, median of 5"}


def _scale_peaks(peaks, mhz_probe, mhz_run):
    """The measured peaks at the clock the timed kernel ran at: the probes'
    rates scaled by (median SM clock in the timed region) / (median SM clock
    during the probes). Unchanged when either clock is unknown."""
    if not mhz_probe or not mhz_run:
        return dict(peaks, clock_scale=1.0)
    k = float(mhz_run) / float(mhz_probe)
    return dict(peaks, fp32_tflops=peaks["fp32_tflops"] * k, mufu_gops=peaks["mufu_gops"] * k, clock_scale=k)


def _alu_roofline(work, ms, peaks, leaf_kind="tri"):
    """Roofline of one traversal launch against the FP32 pipe with the MUFU
    pipe as co-bound: work = per-launch totals of Barnes-Hut tests, far-field
    accepts and exact leaf terms (the kernel's work counts, identical to the
    oracle's); each unit is charged the method's own per-unit cost
    (METHOD_FLOPS / METHOD_MUFU, leaf terms at `leaf_kind`'s cost); ms = the
    launch's duration. frac is the larger of the two pipes' fractions, and
    achieved / peak / unit are that pipe's."""
    t = ms / 1e3
    flops = (work["test"] * METHOD_FLOPS["test"] + work["far"] * METHOD_FLOPS["far"]
             + work["leaf"] * METHOD_FLOPS[leaf_kind])
    mufu = work["far"] * METHOD_MUFU["far"] + work["leaf"] * METHOD_MUFU[leaf_kind]
    fp32 = flops / t / 1e12
    mu = mufu / t / 1e9
    f_fp32, f_mufu = fp32 / peaks["fp32_tflops"], mu / peaks["mufu_gops"]
    fp32_line = {"pipe": "fp32", "achieved": fp32, "peak": peaks["fp32_tflops"], "unit": "TFLOP/s", "frac": f_fp32}
    mufu_line = {"pipe": "mufu", "achieved": mu, "peak": peaks["mufu_gops"], "unit": "Gop/s", "frac": f_mufu}
    bind, co = (fp32_line, mufu_line) if f_fp32 >= f_mufu else (mufu_line, fp32_line)
    return {"bound": "alu", "achieved": bind["achieved"], "peak": bind["peak"], "unit": bind["unit"],
            "frac": bind["frac"], "binding_pipe": bind["pipe"], "co_bound": co,
            "work_per_launch": {"flops": flops, "mufu_ops": mufu, "tests": work["test"], "far_accepts": work["far"],
                                "leaf_terms": work["leaf"], "leaf_kind": leaf_kind},
            "method_costs": {"flops": {k: METHOD_FLOPS[k] for k in ("test", "far", leaf_kind)},
                             "mufu": {k: METHOD_MUFU[k] for k in ("test", "far", leaf_kind)}}}


class _Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons every 50 ms into
    a temporary file. Started before the warm-up (nvidia-smi takes a moment
    to begin); only the samples stamped inside the timed window [mark(),
    stop()] are kept, widened to the nearest sample on each side when the
    window is shorter than the sampling interval. Further named windows
    (begin(name) / end(name), e.g. the pipe probes) are summarised the same
    way in `windows` once stop() has run."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index):
        self.p = None
        self.t0 = None
        self.spans = {}
        self.windows = {}
        fd, self.path = tempfile.mkstemp(prefix="sd_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
            return
        t_end = time.time() + 5.0
        while time.time() < t_end and os.path.getsize(self.path) == 0 and self.p.poll() is None:
            time.sleep(0.02)

    def mark(self):
        self.t0 = time.time()

    def begin(self, name):
        self.spans[name] = [time.time(), None]

    def end(self, name):
        if name in self.spans:
            self.spans[name][1] = time.time()

    @staticmethod
    def _stamp(txt):
        """nvidia-smi's local-time stamp "YYYY/MM/DD hh:mm:ss.fff" in epoch seconds."""
        main, _, frac = txt.partition(".")
        try:
            return time.mktime(time.strptime(main, "%Y/%m/%d %H:%M:%S")) + (float("0." + frac) if frac else 0.0)
        except ValueError:
            return None

    @classmethod
    def _summary(cls, rows, t0, t1):
        inside = [r for r in rows if r[0] is not None and t0 <= r[0] <= t1]
        if not inside:
            before = [r for r in rows if r[0] is not None and r[0] < t0]
            after = [r for r in rows if r[0] is not None and r[0] > t1]
            inside = before[-1:] + after[:1] or rows[-1:]
        reasons = sorted({nm for r in inside for nm, on in zip(cls.REASONS, r[3]) if on})
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "samples": len(inside), "interval_ms": 50, "reasons": reasons}

    def stop(self):
        if self.p is None:
            return None
        t1 = time.time()
        time.sleep(0.1)      # the sample that closes the window
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            ts = self._stamp(parts[0])
            try:
                rows.append((ts, float(parts[2]), float(parts[3]), [v.lower() == "active" for v in parts[6:10]]))
            except ValueError:
                continue
        try:
            os.unlink(self.path)
        except OSError:
            pass
        if not rows:
            return None
        for name, (a, b) in self.spans.items():
            self.windows[name] = self._summary(rows, a, b if b is not None else t1)
        return self._summary(rows, self.t0 if self.t0 is not None else t1, t1)


def _max_over_ranks(ms, device):
    """The slowest rank's time per step; every rank calls it (a no-op
    without a process group)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_value(ms, per_rank_units, world):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * per_rank_units / (ms / 1e3)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2108_10480_gb300 import SmoothDistance, kernel_launches

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    c = _workload(args, rank)
    V = torch.from_numpy(c["V"]).to(dev)
    F = torch.from_numpy(c["F"]).to(dev)
    q = torch.from_numpy(c["queries"]).to(dev)
    M = q.shape[0]
    val = torch.empty(M, device=dev)
    grad = torch.empty(M, 3, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    side = torch.cuda.Stream(device=dev)
    fork, join = torch.cuda.Event(), torch.cuda.Event()
    order = torch.empty(M, dtype=torch.int32, device=dev)

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        fork.record(stream)
        # the build's input checks run on the device and are read back once
        # after the timed region (status below) instead of stalling each step
        sd = SmoothDistance(tris=(V, F), alpha=args.alpha, beta=args.beta, leaf_size=args.leaf_size, device=dev,
                            check=False)
        # the query order on a second stream: it waits for the build's scene
        # box only and overlaps the rest of the build
        side.wait_event(fork)
        sd.query_order(q, stream=side, out=order)
        join.record(side)
        stream.wait_event(join)
        if evs:
            evs[1].record(stream)
        sd.query(q, out=(val, grad), order=order)
        if evs:
            evs[2].record(stream)
        return sd

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = _Clocks(local) if rank == 0 else None
    peaks = _pipe_peaks(dev, clocks) if rank == 0 else None
    for _ in range(max(args.warmup, 0)):
        step()
    # work counts of this workload (decisions are deterministic)
    sd = step()
    _, _, cnt = sd.query(q, counts=True)
    tot = cnt.to(torch.int64).sum(0).tolist()
    del sd
    barrier()
    if clocks:
        clocks.mark()
    launches0 = kernel_launches()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    t_wall = time.perf_counter()
    sd_last = None
    for k in range(args.steps):
        flush.fill_(k & 255)
        sd_last = step(evs[k])
    barrier()
    if sd_last is not None and sd_last.status() != 0:
        raise RuntimeError("the benchmark mesh failed the build's input checks")
    t_wall = time.perf_counter() - t_wall
    launches = kernel_launches() - launches0
    clk = clocks.stop() if clocks else None
    step_ms = [e[0].elapsed_time(e[2]) for e in evs]
    trav_ms = [e[1].elapsed_time(e[2]) for e in evs]
    build_ms = [e[0].elapsed_time(e[1]) for e in evs]
    ms = _max_over_ranks(sum(step_ms) / len(step_ms), dev)
    value = _job_value(ms, M, world)

    out = None
    if rank == 0:
        trav = statistics.mean(trav_ms)
        kh = _src_hash()
        pw = clocks.windows.get("pipe_probes") if clocks else None
        pk = _scale_peaks(peaks, pw and pw["sm_mhz"], clk and clk["sm_mhz"])
        roof = _alu_roofline({"test": tot[0], "far": tot[1], "leaf": tot[2]}, trav, pk, "tri")
        kflops = tot[0] * KERNEL_FLOPS["test"] + tot[1] * KERNEL_FLOPS["far"] + tot[2] * KERNEL_FLOPS["tri"]
        roof.update({"traffic": _traffic(kh), "kernel": "k_traverse<tris,grad>", "kernel_src_hash": kh,
                     "launch_ms": trav,
                     "peak_source": pk["source"] + f"; scaled to the timed region's clock (x{pk['clock_scale']:.4f})",
                     "peaks": {"fp32_tflops": pk["fp32_tflops"], "mufu_gops": pk["mufu_gops"],
                               "probes": peaks["probes"], "probe_clocks": pw},
                     "kernel_count": {"flops_per_launch": kflops, "tflops": kflops / (trav / 1e3) / 1e12,
                                      "frac": kflops / (trav / 1e3) / 1e12 / pk["fp32_tflops"],
                                      "costs": dict(KERNEL_FLOPS),
                                      "what": "the kernel's own hand count of its source (context only)"}})
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded generators, synth/)",
            "config": _config(args, world),
            "breakdown_ms": {"build_and_order": statistics.mean(build_ms), "traverse": trav},
            "work": {"bh_tests": tot[0], "far_accepts": tot[1], "leaf_triangles": tot[2],
                     "per_query": [x / M for x in tot]},
            "roofline": roof,
            "gpu_launches": launches,
            "wall_s_timed": t_wall,
        }
        if clk:
            out["clocks"] = clk
        if not args.no_cells:
            out["cells"] = _cells(args, dev, V, F, q, pk)
        if not args.no_extras:
            out.update(_extras(args, c, V, F, q, dev, M))
    if not args.no_extras:
        # every rank: one body's vertices split across the ranks
        sh = _sharded_pose_leg(dev, rank, world)
        if out is not None:
            out["pose_sharded"] = sh
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return out


def _timed_queries(sd, q, order, val, grad, reps, flush):
    """Median CUDA-event time of one sd_query launch over `reps` launches,
    the L2 flushed (256 MiB write) before each, outside the timed region."""
    import torch
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sd.query(q, out=(val, grad), order=order)
    ts = []
    for k in range(reps):
        flush.fill_(k & 255)
        e0.record(stream)
        sd.query(q, out=(val, grad), order=order)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def _cell_row(sd, q, order, val, grad, flush, peaks, leaf_kind, reps):
    import torch
    M = q.shape[0]
    _, _, cnt = sd.query(q, counts=True, order=order)
    tot = cnt.to(torch.int64).sum(0).tolist()
    ms = _timed_queries(sd, q, order, val, grad, reps, flush)
    roof = _alu_roofline({"test": tot[0], "far": tot[1], "leaf": tot[2]}, ms, peaks, leaf_kind)
    return {"queries": M, "ms": ms, "queries_per_s": M / (ms / 1e3),
            "per_query": {"bh_tests": tot[0] / M, "far_accepts": tot[1] / M, "leaf_terms": tot[2] / M},
            "frac": roof["frac"], "binding_pipe": roof["binding_pipe"],
            "fp32_tflops": roof["achieved"] if roof["binding_pipe"] == "fp32" else roof["co_bound"]["achieved"],
            "mufu_frac": roof["frac"] if roof["binding_pipe"] == "mufu" else roof["co_bound"]["frac"]}


def _cells(args, dev, V, F, q, peaks, reps=5):
    """The traversal (sd_query, value + gradient, Hilbert order computed
    once outside the timing) on every (alpha, beta) cell of the icosphere
    workload (81,920 triangles, 262,144 queries) and on the street point
    queries (the 100,002 vertices of the posed body against 2,000,000 lidar
    points + 50,000 wire segments, alpha 50, beta 0.5): queries/s, the work
    counts per query and the roofline fraction with the method's per-unit
    costs. On the street every leaf term is charged a point's cost (the
    counts do not split points from wire segments; segments cost more, so
    this under-counts the work)."""
    import torch

    from paper_2108_10480_gb300 import SmoothDistance
    from paper_2108_10480_gb300 import pose as gp
    M = q.shape[0]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    val, grad = torch.empty(M, device=dev), torch.empty(M, 3, device=dev)
    rows = []
    for beta in CELL_BETAS:
        for alpha in CELL_ALPHAS:
            sd = SmoothDistance(tris=(V, F), alpha=alpha, beta=beta, leaf_size=args.leaf_size, device=dev)
            order = sd.query_order(q)
            r = _cell_row(sd, q, order, val, grad, flush, peaks, "tri", reps)
            rows.append(dict({"workload": "icosphere-L6", "alpha": alpha, "beta": beta}, **r))
            del sd
    s = _street()
    b = synth.config3_body()
    sd = SmoothDistance(points=s["points"], edges=(s["wire_V"], s["wire_E"]), alpha=50.0, beta=0.5, device=dev)
    X0 = torch.from_numpy(b["V0"]).to(dev)
    X, _, _ = gp.pose_query(sd, X0, np.concatenate([b["theta"], b["p"]]))
    X = X.contiguous()
    vs, gs = torch.empty(X.shape[0], device=dev), torch.empty(X.shape[0], 3, device=dev)
    order = sd.query_order(X)
    r = _cell_row(sd, X, order, vs, gs, flush, peaks, "point", reps)
    rows.append(dict({"workload": "street 2M points + 50k wires, 100,002 body vertices", "alpha": 50.0,
                      "beta": 0.5}, **r))
    return {"what": "sd_query (value + gradient) per cell, median of 5 launches with the L2 flushed before each; "
                    "frac = method work (per-unit costs of the roofline) / launch time / measured pipe peak",
            "rows": rows}


def _extras(args, c, V, F, q, dev, M):
    """plain GPU brute force, end-to-end through host buffers, CPU oracle."""
    import torch

    from paper_2108_10480_gb300 import SmoothDistance
    res = {}
    stream = torch.cuda.current_stream()
    # plain method (all pairs) on the same queries
    sd = SmoothDistance(tris=(V, F), alpha=args.alpha, beta=args.beta, leaf_size=args.leaf_size, device=dev)
    vb = torch.empty(M, device=dev)
    gb = torch.empty(M, 3, device=dev)
    sd.query_brute(q, out=(vb, gb))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sd.query_brute(q, out=(vb, gb))
    e1.record(stream)
    torch.cuda.synchronize()
    tb = e0.elapsed_time(e1)
    res["plain"] = {"value": M / (tb / 1e3), "unit": UNIT, "ms": tb, "what": "sd_query_brute, all pairs"}
    del sd
    # end to end: pinned host inputs -> device, build + order + query, result -> pinned host.
    # The mesh (vertices and faces) travels as one copy and the result (values
    # and gradients) as one: both sides hold them in one buffer each.
    nvb, nfb = V.numel() * 4, F.numel() * 4
    hmesh = torch.empty(nvb + nfb, dtype=torch.uint8).pin_memory()
    hmesh[:nvb].view(torch.float32).copy_(torch.from_numpy(c["V"]).reshape(-1))
    hmesh[nvb:].view(torch.int32).copy_(torch.from_numpy(c["F"]).reshape(-1))
    dmesh = torch.empty(nvb + nfb, dtype=torch.uint8, device=dev)
    dV = dmesh[:nvb].view(torch.float32).view(V.shape)
    dF = dmesh[nvb:].view(torch.int32).view(F.shape)
    hq = torch.from_numpy(c["queries"]).pin_memory()
    dq = torch.empty_like(q)
    hout = torch.empty(4 * M).pin_memory()
    dout = torch.empty(4 * M, device=dev)
    dv, dg = dout[:M], dout[M:].view(M, 3)

    side = torch.cuda.Stream(device=dev)
    meshed, join = torch.cuda.Event(), torch.cuda.Event()
    de = torch.empty(M, dtype=torch.int32, device=dev)

    def e2e_step():
        # mesh upload and build on the main stream; query upload (once the
        # mesh is across, so that the build's input never shares the copy
        # bandwidth) and order on a second one; then the query
        dmesh.copy_(hmesh, non_blocking=True)
        meshed.record(stream)
        s = SmoothDistance(tris=(dV, dF), alpha=args.alpha, beta=args.beta, leaf_size=args.leaf_size, device=dev,
                           check=False)
        side.wait_event(meshed)
        with torch.cuda.stream(side):
            dq.copy_(hq, non_blocking=True)
        s.query_order(dq, stream=side, out=de)
        join.record(side)
        stream.wait_event(join)
        s.query(dq, out=(dv, dg), order=de)
        hout.copy_(dout, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    n = max(3, args.steps)
    e0.record(stream)
    for _ in range(n):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    te = e0.elapsed_time(e1) / n
    res["e2e"] = {"value": M / (te / 1e3), "unit": UNIT, "ms_per_step": te,
                  "h2d_bytes_per_step": int(hmesh.numel() + hq.numel() * 4),
                  "d2h_bytes_per_step": int(hout.numel() * 4)}
    res["cpu_baseline"] = _cpu_baseline(c, args, min_seconds=10.0)
    res["pose"] = _pose_leg(args, dev)
    res["batch"] = _batch_leg(args, dev)
    res["surrogate"] = _surrogate_leg(args, dev)
    res["query_mesh"] = _mesh_leg(args, dev)
    res["sphere_trace"] = _trace_leg(args, dev)
    res["voxel_grid"] = _voxel_leg(args, dev)
    res["beta_switch"] = _switch_leg(args, dev)
    res["rigid"] = _rigid_leg(args, dev)
    return res


def _rigid_leg(args, dev, steps=8, h=0.005):
    """Rigid-body time steps (Sec. 4.5, Eq. opt) of the 100,002-vertex body
    against the street (2,000,000 points + 50,000 wires, alpha 50, beta 0.5,
    alpha_q 100): the body starts where D = 2 cm, moving at (0.5, 0, -3) m/s
    under gravity; each step is the interior-point solve, every constraint
    evaluation one placement + query + reduction on the GPU."""
    import torch

    from paper_2108_10480_gb300 import SmoothDistance
    from paper_2108_10480_gb300.rigid import RigidBody
    s = _street()
    b = synth.config3_body()
    sd = SmoothDistance(points=s["points"], edges=(s["wire_V"], s["wire_E"]), alpha=50.0, beta=0.5, device=dev)
    X0 = torch.from_numpy(b["V0"]).to(dev)
    ax = np.array([2.0, 1.0, 0.7])
    I_body = np.diag([(ax[1] ** 2 + ax[2] ** 2), (ax[0] ** 2 + ax[2] ** 2), (ax[0] ** 2 + ax[1] ** 2)]) / 5.0
    body = RigidBody(sd, X0, 1.0, I_body, b["theta"], b["p"], v=(0.5, 0.0, -3.0))
    lo, hi = float(b["p"][2]) - 3.0, float(b["p"][2]) + 3.0
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        D = body.constraint(np.concatenate([body.theta, [body.p[0], body.p[1], mid]]), 100.0)[0]
        lo, hi = (lo, mid) if D > 0.02 else (mid, hi)
    body.p[2] = hi
    rows = []
    t0 = time.perf_counter()
    for _ in range(steps):
        ts = time.perf_counter()
        info = body.step(h, (0.0, 0.0, -9.81), 100.0, max_iter=200)
        torch.cuda.synchronize()
        rows.append(dict(info, ms=1e3 * (time.perf_counter() - ts), D=float(info["D"]), lam=float(info["lambda"])))
    total = time.perf_counter() - t0
    ev = sum(r["evaluations"] for r in rows)
    return {"what": "rigid time steps (h 5 ms) of the 100,002-vertex body falling onto the street; IPM with "
                    "identity Hessian, constraint on the GPU", "steps": rows, "ms_per_step": 1e3 * total / steps,
            "evaluations_per_step": ev / steps, "ms_per_evaluation": 1e3 * total / ev,
            "min_D": min(r["D"] for r in rows)}


def _unit_box(X):
    """Scale and translate so the bounding box is centred at (0.5, 0.5, 0.5)
    with diagonal 0.5 (the voxel benchmark's normalisation)."""
    X = np.asarray(X, np.float64)
    lo, hi = X.min(0), X.max(0)
    return ((X - 0.5 * (lo + hi)) * (0.5 / np.linalg.norm(hi - lo)) + 0.5).astype(np.float32)


def _voxel_leg(args, dev):
    """The performance benchmark of Sec. 4.4 on synthetic meshes (bumpy
    spheres and tori, 80 to 81,920 triangles) in place of Thingi10K: each
    mesh as its vertices V, edges E and triangles F, scaled into a box of
    diagonal 0.5 centred in the unit cube; d^ and its gradient at the
    1,000,000 voxel centres of a 100^3 grid over [0, 1]^3, beta 0.5, alpha
    by the paper's heuristic (1 / shortest edge for E and F, 100 x the
    bounding-box diagonal for V). Leaves visited = exact primitive terms +
    far-field expansions per query."""
    import torch

    from paper_2108_10480_gb300 import SmoothDistance
    g = (np.arange(100) + 0.5) / 100
    q = torch.from_numpy(np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)).to(dev)
    M = q.shape[0]
    meshes = [("blob", lvl) + synth.blob(level=lvl, diag=1.0, seed=10 + lvl) for lvl in (1, 2, 3, 4, 5, 6)]
    meshes += [("torus", n) + synth.torus(n, max(6, n // 3), 1.0, 0.3) for n in (12, 40, 120, 360)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    rows = []
    for name, size, V, F in meshes:
        V = _unit_box(V)
        E = synth.mesh_edges(F)
        emin = float(np.linalg.norm(V[E[:, 0]] - V[E[:, 1]], axis=1).min())
        for kind, kw, alpha in (("V", dict(points=V), 100 * 0.5), ("E", dict(edges=(V, E)), 1.0 / emin),
                                ("F", dict(tris=(V, F)), 1.0 / emin)):
            sd = SmoothDistance(alpha=alpha, beta=0.5, device=dev, **kw)
            sd.query(q)
            torch.cuda.synchronize()
            e0.record(stream)
            sd.query(q)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            _, _, cnt = sd.query(q, counts=True)
            leaves = (cnt[:, 1] + cnt[:, 2]).to(torch.float64)
            n = int(sd.info()["n_prims"])
            rows.append({"mesh": f"{name}-{size}", "kind": kind, "n_prims": n, "alpha": alpha, "ms": ms,
                         "queries_per_s": M / (ms / 1e3), "leaves_visited_mean": float(leaves.mean()),
                         "leaves_visited_max": int(leaves.max()),
                         "leaves_visited_pct_mean": float(100.0 * leaves.mean() / n)})
    return {"what": "100^3 voxel centres, d^ + gradient, beta 0.5, synthetic meshes as V / E / F "
                    "(box diagonal 0.5 in the unit cube)", "rows": rows}


def _switch_leg(args, dev, iso=0.1, probes=4096, dz=2e-3, steps=400):
    """The beta sensitivity study of Sec. 4.3 on the street (2,000,000 points,
    alpha 50): vertical rays from uniform points on the top and bottom of the
    scene box are sphere-traced (in z) down or up to the d^ = 0.1 isosurface;
    from there short vertical marches of 2 mm steps look for points where the
    Barnes-Hut work of beta = 0.5 changes (the evaluation enters a node it
    took as a far field before); at each such point where beta = 0.5001
    traverses less of the tree, the values and gradients of the two betas are
    compared."""
    import torch

    from paper_2108_10480_gb300 import SmoothDistance
    s = _street()
    P = s["points"]
    sd0 = SmoothDistance(points=P, alpha=50.0, beta=0.5, device=dev)
    sd1 = SmoothDistance(points=P, alpha=50.0, beta=0.5001, device=dev)
    lo, hi = P.min(0), P.max(0)
    rng = np.random.default_rng(31)
    xy = lo[:2] + (hi[:2] - lo[:2]) * rng.random((probes, 2))
    top = rng.random(probes) < 0.5
    z = np.where(top, hi[2] + 1.0, lo[2] - 1.0)
    sgn = np.where(top, -1.0, 1.0)
    pts = torch.from_numpy(np.stack([xy[:, 0], xy[:, 1], z], 1).astype(np.float32)).to(dev)
    dirz = torch.from_numpy(sgn.astype(np.float32)).to(dev)
    alive = torch.ones(probes, dtype=torch.bool, device=dev)
    done = torch.zeros(probes, dtype=torch.bool, device=dev)
    zlim = float(hi[2] - lo[2]) + 3.0
    travel = torch.zeros(probes, device=dev)
    for _ in range(200):
        idx = torch.nonzero(alive & ~done).squeeze(1)
        if idx.numel() == 0:
            break
        v, _ = sd0.query(pts[idx], grad=False)
        hit = v <= iso
        done[idx[hit]] = True
        step = v.clamp_min(0) - iso + 1e-4
        move = idx[~hit]
        pts[move, 2] += dirz[move] * step[~hit]
        travel[move] += step[~hit]
        alive[move[travel[move] > zlim]] = False
    start = pts[done]
    dz_t = dirz[done]
    found = []
    prev = None
    for k in range(steps):
        x = start.clone()
        x[:, 2] += dz_t * dz * k
        _, _, c0 = sd0.query(x, counts=True)
        if prev is not None:
            sw = torch.nonzero((c0 != prev).any(1)).squeeze(1)
            if sw.numel():
                found.append(x[sw])
        prev = c0
    if not found:
        return {"what": "beta 0.5 vs 0.5001 at far/near switch points", "points": 0}
    X = torch.cat(found)
    v0, g0, c0 = sd0.query(X, counts=True)
    v1, g1, c1 = sd1.query(X, counts=True)
    less = c1[:, 0] < c0[:, 0]
    dv = (v1 - v0).abs()[less].double()
    cos = torch.nn.functional.cosine_similarity(g0[less], g1[less], dim=1).double()
    return {"what": "street points, alpha 50: d^ = 0.1 isosurface reached by vertical sphere tracing, then "
                    "2 mm vertical marches; points where beta 0.5's traversal changes and beta 0.5001 tests fewer "
                    "nodes", "rays_reaching_isosurface": int(done.sum()), "switch_points": int(X.shape[0]),
            "points_compared": int(less.sum()),
            "value_discrepancy": {"mean": float(dv.mean()) if dv.numel() else None,
                                  "max": float(dv.max()) if dv.numel() else None},
            "gradient_cosine": {"mean": float(cos.mean()) if cos.numel() else None,
                                "min": float(cos.min()) if cos.numel() else None}}


def _trace_leg(args, dev, betas=(0.1, 0.2, 0.3, 0.5, 0.75, 1.0)):
    """The paper's beta study (Sec. 4.3, parameter analysis) on a synthetic
    stand-in for a desktop scan: a bumpy closed mesh of 20,480 triangles
    (10,242 vertices, 30,720 edges, bounding-box diagonal 0.25 m) taken as its
    vertices, its edges or its triangles; alpha 200, alpha_U 1200. Time to
    sphere-trace a 512 x 512 image at each beta (beta = 0, the exact render,
    timed once without a warm-up run), and the isosurface error
    |depth(beta) - depth(0)| / diagonal over the rays that hit at both."""
    import torch

    from paper_2108_10480_gb300 import SmoothDistance
    V, F = synth.blob(level=5)
    E = synth.mesh_edges(F)
    cam = synth.trace_camera(V, 512, 512)
    t_max = 4.0 * cam["diag"]
    out = {"what": "512x512 sphere-traced renders of a 20,480-triangle bumpy mesh (diag 0.25 m) as vertices, "
                   "edges or triangles, alpha 200, alpha_U 1200, eps 1e-5 m; error vs the beta = 0 render",
           "kinds": {}}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()

    def timed(sd, warm):
        if warm:
            sd.sphere_trace(cam, eps=1e-5, t_max=t_max)
        torch.cuda.synchronize()
        e0.record(stream)
        d, _, ev = sd.sphere_trace(cam, eps=1e-5, t_max=t_max)
        e1.record(stream)
        torch.cuda.synchronize()
        return d.cpu().numpy(), ev, e0.elapsed_time(e1)
    for kind, kw in (("vertices", dict(points=V)), ("edges", dict(edges=(V, E))), ("triangles", dict(tris=(V, F)))):
        d0, ev0, ms0 = timed(SmoothDistance(alpha=200.0, alpha_u=1200.0, beta=0.0, device=dev, **kw), False)
        rows = [{"beta": 0.0, "ms_512": ms0, "evaluations": ev0, "evals_per_s": ev0 / (ms0 / 1e3),
                 "err_mean_rel_diag": 0.0, "err_max_rel_diag": 0.0, "hit_mismatch_frac": 0.0}]
        for beta in betas:
            db, ev, ms = timed(SmoothDistance(alpha=200.0, alpha_u=1200.0, beta=beta, device=dev, **kw), True)
            both = np.isfinite(d0) & np.isfinite(db)
            err = np.abs(db[both] - d0[both]) / cam["diag"]
            rows.append({"beta": beta, "ms_512": ms, "evaluations": ev, "evals_per_s": ev / (ms / 1e3),
                         "err_mean_rel_diag": float(err.mean()), "err_max_rel_diag": float(err.max()),
                         "hit_mismatch_frac": float((np.isfinite(d0) != np.isfinite(db)).mean())})
        out["kinds"][kind] = rows
    return out


def _mesh_leg(args, dev, reps=10):
    """Triangle queries (Sec. 3.4) and the query-mesh objective (Sec. 3.6) on
    the street (2,000,000 points + 50,000 wire segments, alpha 50, beta 0.5):
    the 200,000 triangles of the posed 100,002-vertex body as query
    primitives; one evaluation = sd_query_prims (value + translation
    gradient per triangle) + sd_mesh_reduce (D, alpha_q = 100, and the
    per-vertex gradients). Also the triangles' work counts."""
    import torch

    from paper_2108_10480_gb300 import SmoothDistance, mesh_reduce
    s = _street()
    b = synth.config3_body()
    R = _rotation(b["theta"])
    Vq = (b["V0"].astype(np.float64) @ R.T + b["p"]).astype(np.float32)
    sd = SmoothDistance(points=s["points"], edges=(s["wire_V"], s["wire_E"]), alpha=50.0, beta=0.5, device=dev)
    Vt = torch.from_numpy(Vq).to(dev)
    Ft = torch.from_numpy(b["F"].astype(np.int32)).to(dev)
    m = Ft.shape[0]
    val = torch.empty(m, device=dev)
    grad = torch.empty(m, 3, device=dev)

    def one():
        sd.query_prims(Vt, Ft, out=(val, grad))
        return mesh_reduce(Ft, Vt.shape[0], val, grad, 100.0)
    for _ in range(3):
        one()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        D, vg = one()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    _, _, cnt = sd.query_prims(Vt, Ft, counts=True)
    per = cnt.to(torch.float64).mean(0).tolist()
    return {"what": "street, the posed 100,002-vertex body's 200,000 triangles as queries: "
                    "sd_query_prims + sd_mesh_reduce (alpha_q 100)",
            "triangles": m, "ms_per_evaluation": ms, "value": m / (ms / 1e3), "unit": "triangle queries/s",
            "D": float(D.item()), "work_per_triangle": {"bh_tests": per[0], "far_accepts": per[1], "leaf_prims": per[2]},
            "status": sd.status()}


def _rotation(theta):
    """Rotation matrix of a rotation vector (Rodrigues)."""
    th = np.asarray(theta, np.float64)
    t = float(np.linalg.norm(th))
    K = np.array([[0.0, -th[2], th[1]], [th[2], 0.0, -th[0]], [-th[1], th[0], 0.0]])
    if t < 1e-12:
        return np.eye(3) + K
    return np.eye(3) + np.sin(t) / t * K + (1 - np.cos(t)) / (t * t) * K @ K


def _surrogate_leg(args, dev, reps=3):
    """Learned far-field surrogate on the street (2,000,000 points + 50,000
    wire segments, alpha 50, beta 0.5): the network is trained by the
    library's kernels on Barnes-Hut values of 10M uniform samples of the
    scene box padded by 5 m (those whose certified bound exceeds 0.5 m, the
    region where it can be routed), then 16M mixed queries (half uniform in
    the padded box, half within ~1 m of the lidar points) are answered with
    LB > margin routed to LB + the network (trained on the residual over
    LB) and the rest to the traversal; value + gradient, compared with the
    traversal alone on the same queries. Swept: two training budgets (3 and
    10 epochs over the same samples) x routing margins 1, 2 and 5 m, each
    reporting its speed-up over the traversal alone and the routed answers'
    errors (the traversal's value as reference)."""
    import torch

    from paper_2108_10480_gb300 import SmoothDistance
    from paper_2108_10480_gb300.surrogate import Surrogate, lower_bound
    s = _street()
    sd = SmoothDistance(points=s["points"], edges=(s["wire_V"], s["wire_E"]), alpha=50.0, beta=0.5, device=dev)
    lo = np.minimum(s["points"].min(0), s["wire_V"].min(0)) - 5.0
    hi = np.maximum(s["points"].max(0), s["wire_V"].max(0)) + 5.0
    t0 = time.perf_counter()
    xs = torch.from_numpy(synth.uniform_box(10_000_000, lo, hi, 21)).to(dev)
    lbs, _, far = lower_bound(sd, xs, margin=0.5, grad=False)
    xs = xs[far.bool()].contiguous()
    ts, _ = sd.query(xs, grad=False)
    torch.cuda.synchronize()
    label_s = time.perf_counter() - t0
    scale = float((ts - lbs[far.bool()]).abs().max())
    del lbs
    n = 16 * 1024 * 1024
    rng = np.random.default_rng(22)
    near = s["points"][rng.integers(0, s["points"].shape[0], n // 2)] + \
        rng.normal(0.0, 0.6, (n // 2, 3)).astype(np.float32)
    q = torch.from_numpy(np.concatenate([synth.uniform_box(n - n // 2, lo, hi, 23), near])).to(dev)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    vb, gb = torch.empty(n, device=dev), torch.empty(n, 3, device=dev)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_bh = timed(lambda: sd.query(q, out=(vb, gb)))
    sweep = []
    default = None
    for epochs in (3, 10):
        t1 = time.perf_counter()
        sur = Surrogate(lo, hi, sigma=12.0, seed=1, scale=scale, device=dev)
        hist = sur.fit_residual(sd, xs, ts, epochs=epochs, batch=4096, lr=1e-3)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t1
        for margin in (1.0, 2.0, 5.0):
            res = {}

            def routed():
                res["out"] = sur.query(sd, q, margin=margin)
            ms_sur = timed(routed)
            v, g, r, nr = res["out"]
            rb = r.bool()
            err = (v[rb] - vb[rb]).abs()
            gerr = (g[rb] - gb[rb]).norm(dim=1)
            row = {"epochs": epochs, "margin_m": margin, "train_s": train_s, "loss_last_epoch": hist[-1],
                   "routed_fraction": nr / n, "ms_routed": ms_sur, "speedup": ms_bh / ms_sur,
                   "abs_err_m": {"p50": _pct(err, 0.5), "p99": _pct(err, 0.99),
                                 "max": float(err.max().item()) if err.numel() else None},
                   "grad_err": {"p50": _pct(gerr, 0.5), "p99": _pct(gerr, 0.99)}}
            sweep.append(row)
            if epochs == 3 and margin == 1.0:
                default = (sur, row, rb, res["out"])
    sur, row, rb, (v, g, r, nr) = default
    qr = q[rb].contiguous()
    ms_mlp = timed(lambda: sur.forward(qr))
    ms_lb = timed(lambda: lower_bound(sd, q, margin=1.0))
    lbq, _, _ = lower_bound(sd, q, margin=1.0, grad=False)
    err_lb = (lbq[rb] - vb[rb]).abs()
    return {"what": "street, 16M mixed queries (8M uniform in the box padded by 5 m, 8M near the points); "
                    "LB > margin -> LB + MLP, else Barnes-Hut; value + gradient; sweep of training budget x margin",
            "train": {"samples": int(far.sum().item()), "label_s": label_s, "batch": 4096},
            "ms_barnes_hut": ms_bh, "sweep": sweep,
            "routed_fraction": row["routed_fraction"], "ms_routed": row["ms_routed"], "speedup": row["speedup"],
            "value": n / (row["ms_routed"] / 1e3), "unit": "queries/s", "ms_lower_bound_all": ms_lb,
            "mlp_forward": {"queries": nr, "ms": ms_mlp, "queries_per_s": nr / (ms_mlp / 1e3),
                            "tflops": nr * MLP_FLOPS / (ms_mlp / 1e3) / 1e12, "flops_per_query": MLP_FLOPS,
                            "roofline": _tensor_roofline(nr * MLP_FLOPS / (ms_mlp / 1e3) / 1e12)},
            "abs_err_m": row["abs_err_m"], "grad_err": row["grad_err"],
            "lb_alone_abs_err_m": {"p50": _pct(err_lb, 0.5), "p99": _pct(err_lb, 0.99)}}


def _pct(x, p):
    if x.numel() == 0:
        return None
    xs = x.sort().values
    return float(xs[int(p * (x.numel() - 1))].item())


def _batch_leg(args, dev, reps=10):
    """64 rigid bodies (icospheres/tori, 1k-200k vertices each, 2,816,048 in
    total) against the street (2,000,000 points + 50,000 wire segments,
    alpha 50, beta 0.5), outer LSE alpha_q = 100 per body: one evaluation =
    placement + ordering + ONE persistent traversal + per-body reductions,
    replayed from a CUDA graph, block size and leaf size from the autotuner;
    compared with the plain per-body loop (sd_pose_query + sd_pose_reduce,
    leaf size 1, default block) on the same data."""
    import torch

    from paper_2108_10480_gb300 import SmoothDistance
    from paper_2108_10480_gb300 import pose as gp
    from paper_2108_10480_gb300.batch import BatchedBodies, autotune
    s = _street()
    bl = synth.config4_bodies()
    bodies = [b["V0"] for b in bl]
    poses = np.array([np.concatenate([b["theta"], b["p"]]) for b in bl])
    M = int(sum(b.shape[0] for b in bodies))
    kw = dict(points=s["points"], edges=(s["wire_V"], s["wire_E"]), alpha=50.0, beta=0.5, device=dev)
    lo, hi = s["points"].min(0), s["points"].max(0)
    sample = synth.uniform_box(1024, lo, hi, 11)
    t0 = time.perf_counter()
    best, recs = autotune(kw, bodies, poses, 100.0, sample, leaf_sizes=(1, 2, 4), blocks=(64, 128, 256), reps=3)
    tune_s = time.perf_counter() - t0
    sd = SmoothDistance(leaf_size=best["leaf_size"], **kw)
    bb = BatchedBodies(sd, bodies)
    bb.block = best["block"]
    bb.set_poses(poses)
    g = bb.capture(100.0)
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    # plain: one body at a time through the single-body API, leaf size 1
    sd1 = SmoothDistance(leaf_size=1, **kw)
    X0s = [torch.from_numpy(b).to(dev) for b in bodies]

    def plain():
        for X0, ps in zip(X0s, poses):
            X, v, gr = gp.pose_query(sd1, X0, ps)
            gp.pose_reduce(X0, v, gr, ps, alpha_q=100.0)
    plain()
    torch.cuda.synchronize()
    e0.record()
    plain()
    e1.record()
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1)
    return {"what": f"64 bodies, {M} vertices vs the street; graph-replayed batch (autotuned) vs per-body loop",
            "autotune": {"best": best, "candidates": recs, "seconds": tune_s},
            "ms_per_evaluation": ms, "value": M / (ms / 1e3), "unit": "vertex queries/s",
            "plain_per_body_loop": {"ms": ms_plain, "value": M / (ms_plain / 1e3)},
            "speedup_vs_plain": ms_plain / ms}


def _pose_leg(args, dev, iters=20):
    """Rigid-body constraint on the street workload: 2,000,000 lidar points +
    50,000 wire segments (alpha 50, beta 0.5), a 100,002-vertex body, outer
    LogSumExp alpha_q = 100; one evaluation = placement + Barnes-Hut query of
    every vertex + outer LSE + pose gradient (sd_pose_query + sd_pose_reduce)."""
    import torch

    from paper_2108_10480_gb300 import SmoothDistance
    from paper_2108_10480_gb300 import pose as gp
    s = _street()
    b = synth.config3_body()
    P = torch.from_numpy(s["points"]).to(dev)
    Vw = torch.from_numpy(s["wire_V"]).to(dev)
    Ew = torch.from_numpy(s["wire_E"]).to(dev)
    X0 = torch.from_numpy(b["V0"]).to(dev)
    pose = np.concatenate([b["theta"], b["p"]])
    stream = torch.cuda.current_stream()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    for _ in range(2):
        sd = SmoothDistance(points=P, edges=(Vw, Ew), alpha=50.0, beta=0.5, device=dev)
    torch.cuda.synchronize()
    e0.record(stream)
    sd = SmoothDistance(points=P, edges=(Vw, Ew), alpha=50.0, beta=0.5, device=dev)
    e1.record(stream)
    torch.cuda.synchronize()
    build_ms = e0.elapsed_time(e1)
    for _ in range(3):
        X, v, g = gp.pose_query(sd, X0, pose)
        gp.pose_reduce(X0, v, g, pose, alpha_q=100.0)
    torch.cuda.synchronize()
    e1.record(stream)
    for _ in range(iters):
        X, v, g = gp.pose_query(sd, X0, pose)
        out, _ = gp.pose_reduce(X0, v, g, pose, alpha_q=100.0)
    e2.record(stream)
    torch.cuda.synchronize()
    ms = e1.elapsed_time(e2) / iters
    M = X0.shape[0]
    return {"what": "street: 2,000,000 points + 50,000 wire segments, 100,002-vertex body; "
                    "placement + BH query + outer LSE + 6-DoF pose gradient",
            "build_ms": build_ms, "ms_per_evaluation": ms, "value": M / (ms / 1e3), "unit": "vertex queries/s",
            "D": float(out[0].item())}


def _sharded_pose_leg(dev, rank, world, iters=20):
    """One body split across the ranks (strong scaling of a single
    constraint): the 100,002-vertex body against the street (2,000,000
    points + 50,000 wires, alpha 50, beta 0.5, alpha_q 100); each rank places
    and queries its contiguous slice of the vertices, forms its shard's
    partial (sd_pose_partial), and the partials are all-gathered (9 floats
    per rank, the only exchange) and merged on the host (sd_pose_merge). The
    result is compared with sd_pose_reduce over the whole body on this
    rank."""
    import torch

    from paper_2108_10480_gb300 import SmoothDistance
    from paper_2108_10480_gb300 import pose as gp
    s = _street()
    b = synth.config3_body()
    pose = np.concatenate([b["theta"], b["p"]])
    sd = SmoothDistance(points=s["points"], edges=(s["wire_V"], s["wire_E"]), alpha=50.0, beta=0.5, device=dev)
    X0 = torch.from_numpy(b["V0"]).to(dev)
    M = X0.shape[0]
    a, e = rank * M // world, (rank + 1) * M // world
    mine = X0[a:e].contiguous()

    def one():
        _, v, g = gp.pose_query(sd, mine, pose)
        part = gp.pose_partial(mine, v, g, pose, alpha_q=100.0)
        return gp.reduce_shards(part, pose, alpha_q=100.0)
    for _ in range(3):
        r = one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(iters):
        r = one()
    ms = 1e3 * (time.perf_counter() - t0) / iters
    ms = _max_over_ranks(ms, dev)
    _, v, g = gp.pose_query(sd, X0, pose)
    whole, _ = gp.pose_reduce(X0, v, g, pose, alpha_q=100.0)
    whole = whole.cpu().numpy().astype(np.float64)
    return {"what": "100,002-vertex body split over the ranks: per-rank placement + BH query + shard partial, "
                    "9-float all-gather, host merge (host wall clock per evaluation, max over ranks)",
            "ranks": world, "vertices_per_rank": e - a, "ms_per_evaluation": ms,
            "value": M / (ms / 1e3), "unit": "vertex queries/s", "D": float(r[0]),
            "rel_diff_vs_whole_body_reduce": {
                "D": float(abs(r[0] - whole[0]) / max(abs(whole[0]), 1e-2)),
                "gradient": float(np.linalg.norm(r[1:] - whole[1:]) / max(np.linalg.norm(whole[1:]), 1e-2))}}


def _cpu_baseline(c, args, sample=None, min_seconds=0.0, single_thread=True):
    """The FP64 oracle as it stands on this host's cores: its own tree build
    over the full mesh plus Barnes-Hut on a query sample (repeated until
    min_seconds of work); the rate is scaled to the full batch as
    M / (t_build + t_query * M / sample). With single_thread, also the same
    Barnes-Hut on one thread over the first 8,192 queries (tree build
    excluded)."""
    import oracle
    cores = oracle.default_threads()
    M = c["queries"].shape[0]
    if sample is None:
        sample = M
    qs = c["queries"][:sample]
    tb = tq = 0.0
    reps = 0
    t_start = time.perf_counter()
    while reps == 0 or time.perf_counter() - t_start < min_seconds:
        t0 = time.perf_counter()
        sc = oracle.Scene(tri_V=c["V"], tri_F=c["F"])
        sc.build_tree(args.leaf_size)
        t1 = time.perf_counter()
        sc.bh(qs, args.alpha, args.beta, threads=cores)
        t2 = time.perf_counter()
        tb += t1 - t0
        tq += t2 - t1
        reps += 1
    tb /= reps
    tq /= reps
    full = tb + tq * M / sample
    out = {"value": M / full, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{reps} x (oracle tree build over all 81,920 triangles ({tb:.2f} s) + FP64 Barnes-Hut on "
                     f"{'all' if sample == M else f'the first {sample} of'} {M} queries ({tq:.2f} s, {cores} "
                     f"threads)); mean per pass" + ("" if sample == M else ", rate scaled to the full batch")}
    if single_thread:
        n1 = min(8192, M)
        t0 = time.perf_counter()
        sc.bh(c["queries"][:n1], args.alpha, args.beta, threads=1)
        t1 = time.perf_counter() - t0
        out["single_thread"] = {"value": n1 / t1, "unit": UNIT, "cores": 1,
                                "sample": f"FP64 Barnes-Hut on the first {n1} queries, one thread, tree prebuilt "
                                          f"({t1:.2f} s)"}
    return out


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, each step a bounded
    sample of the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import oracle
    c = _workload(args, 0)
    cores = oracle.default_threads()
    M = c["queries"].shape[0]
    times = []
    for k in range(args.warmup + args.steps):
        r = _cpu_baseline(c, args, sample=M, single_thread=False)
        if k >= args.warmup:
            times.append(M / r["value"])
    ms = 1e3 * sum(times) / len(times)
    value = M / (ms / 1e3)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generators, synth/)",
            "config": _config(args, args.gpus), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"per step: oracle tree build over all 81,920 triangles + FP64 "
                                       f"Barnes-Hut on all {M} queries ({cores} threads), measured"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = _args()
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
