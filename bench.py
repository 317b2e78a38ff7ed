"""Benchmark of the all-pairs Stokesian-dynamics hot path on GB300.

One JSON line on rank 0.  A step is one explicit Euler step (Sec. 3.1) of the
N = 65,536 system at volume fraction 0.05 with per-particle N(0,1) forces,
float32 inputs, RPY tensor, FP32-compensated pair sums, FP64 positions:
Verlet-list check + FP32 mirror, then the all-pairs kernel beside the list rebuild
(when due) and the FP64 near terms, then the split reduction with the self term
and the Euler update.  value = N^2 pair interactions per second (self pairs
included, as the paper counts them).

Extra legs on rank 0 (reported in the same line): the plain FP64 GPU path on the
same system, the batched workload (16,384 clusters, N per cluster U{4..256}),
the Oseen variant and the CPU oracle on a bounded sample (cpu_baseline); on a
single GPU also the other workloads (four spheres, drift, adjoint), the N sweep,
the paper's fcc benchmark and the lubrication lattice.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank steps its own replica (weak scaling, no collective on
the data path); the elapsed time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RPY pair-interactions/s at N=65536 (FP32-comp vs FP64), batched steps/s"
UNIT = "pair-interactions/s"
N_MAIN = 65536
PHI = 0.05
DT = 0.01
FLOPS_PER_PAIR = 34          # RPY pair term: 3 FADD, 7 FMUL, 12 FFMA (FMA = 2 flops), plus one rsqrt
FP32_LANES_PER_SM = 128
L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.f is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                p = [s.strip() for s in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(s):
            try:
                return float(s)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = [nm for k, nm in enumerate(names) if any(r[5 + k] == "Active" for r in rows)]
        loaded = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(rows), "reasons": reasons}


def _flush_l2(buf):
    buf.add_(1)


def _time_steps(step, nsteps, stream, flush_buf):
    """Sum of CUDA-event durations of `nsteps` calls of step(), each preceded by an
    L2 flush outside the events."""
    import torch
    total = 0.0
    evs = []
    for _ in range(nsteps):
        _flush_l2(flush_buf)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    for e0, e1 in evs:
        total += e0.elapsed_time(e1)
    return total


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


KERNEL_SOURCES = ["dense.cu", "pair.cuh", "ptx.cuh", "sd_internal.h"]
DENSE_PROFILES = {"directed": os.path.join(ROOT, "profiles", "dense2_kernel_N65536_fp32c.md"),
                  "symmetric": os.path.join(ROOT, "profiles", "dense_sym_kernel_N65536_fp32c.md")}
DENSE_NAMES = {"directed": "dense2_kernel<RP, FP32C> (packed f32x2, every ordered pair)",
               "symmetric": "dense_sym_kernel<RP, FP32C> (packed f32x2, each unordered pair once)"}


def _dense_traffic(kind):
    """DRAM bytes per launch of the all-pairs kernel from the committed ncu summary,
    or None when the kernel sources changed since those counters were taken."""
    import hashlib
    import re
    try:
        txt = open(DENSE_PROFILES[kind]).read()
        want = re.search(r"kernel_sources_sha256_16 = ([0-9a-f]+)", txt).group(1)
        val = int(re.search(r"traffic_bytes_per_launch = ([0-9]+)", txt).group(1))
    except (OSError, AttributeError):
        return None
    hsh = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1205_6333_gb300", "csrc", f), "rb") as fh:
            hsh.update(fh.read())
    return val if hsh.hexdigest()[:16] == want else None


def _main_inputs(n):
    from paper_1205_6333_gb300 import inputs
    x, L = inputs.cube_rsa(n, PHI, inputs.SEED_BASE + 2)
    F = inputs.normal_forces(n, inputs.SEED_BASE + 1002)
    return x.astype(np.float32).astype(np.float64), F.astype(np.float32).astype(np.float64), L


def cpu_baseline(x, F, target_s=10.0):
    """The FP64 oracle as it stands, on all host cores, on a bounded row sample of
    the same system; pairs/s scaled from the sample."""
    import oracle
    n = x.shape[0]
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(123)
    rows = rng.choice(n, 128, replace=False).astype(np.int32)
    t0 = time.perf_counter()
    oracle.mobility_rows(x, F, rows, "rpy", nthreads=cores)
    t1 = time.perf_counter()
    rate = len(rows) * n / max(t1 - t0, 1e-6)
    nrows = int(min(n, max(128, target_s * rate / n)))
    rows = rng.choice(n, nrows, replace=False).astype(np.int32)
    t0 = time.perf_counter()
    oracle.mobility_rows(x, F, rows, "rpy", nthreads=cores)
    dt = time.perf_counter() - t0
    # the same loop on one core, on a smaller sample (about a second)
    rows1 = rng.choice(n, max(8, min(n, int(rate / max(cores, 1) / n))), replace=False).astype(np.int32)
    t0 = time.perf_counter()
    oracle.mobility_rows(x, F, rows1, "rpy", nthreads=1)
    dt1 = time.perf_counter() - t0
    return {"value": nrows * n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d of %d rows of the N=%d apply (RPY, FP64, ascending-j loop, OpenMP over rows); %.1f s"
                      % (nrows, n, n, dt),
            "value_one_core": len(rows1) * n / dt1,
            "sample_one_core": "%d rows on 1 thread; %.2f s" % (len(rows1), dt1)}


def _config(L, world):
    return {"workload": "rpy_euler_step_N65536_phi0.05_cube_fp32c", "n": N_MAIN, "phi": PHI,
            "box_side": L, "tensor": "rpy", "precision": "fp32 pair terms, compensated sums, fp64 state",
            "step": "Verlet check + mirror; all-pairs kernel beside (list rebuild when due, fp64 near terms); "
                    "reduction + self, Euler", "dt": DT,
            "l2": "flushed (512 MiB write) before every timed step",
            "parallelism": "replicas" if world > 1 else "single"}


def run_reference(args):
    """--impl reference: the CPU oracle timed on the host cores, same metric/config."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    oracle.build()
    x, F, L = _main_inputs(N_MAIN)
    cores = os.cpu_count() or 1
    rows_per_step = 2048
    rng = np.random.default_rng(7)
    for _ in range(args.warmup):
        r = rng.choice(N_MAIN, 64, replace=False).astype(np.int32)
        oracle.mobility_rows(x, F, r, "rpy", nthreads=cores)
    t = 0.0
    for _ in range(args.steps):
        r = rng.choice(N_MAIN, rows_per_step, replace=False).astype(np.int32)
        t0 = time.perf_counter()
        oracle.mobility_rows(x, F, r, "rpy", nthreads=cores)
        t += time.perf_counter() - t0
    pairs = args.steps * rows_per_step * N_MAIN
    val = pairs / t
    sample = ("each step: %d seeded rows of the N=%d apply (RPY, FP64 oracle, %d threads)"
              % (rows_per_step, N_MAIN, cores))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": _config(L, 1),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import paper_1205_6333_gb300 as sd

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local % torch.cuda.device_count())
        # NCCL between GPUs; SD_BENCH_BACKEND=gloo runs the same multi-rank logic with the
        # exchange staged through host memory (e.g. several ranks sharing one GPU)
        dist.init_process_group(os.environ.get("SD_BENCH_BACKEND", "nccl"))
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    x, F, L = _main_inputs(N_MAIN)
    n = N_MAIN
    s = sd.System(n, prec="fp32c", tensor="rpy", stream="torch", torch_allocator=True, device=dev,
                  dense=args.dense)
    s.set_positions(x)
    s.set_forces(F)
    step = lambda: s.step(DT, 1)   # noqa: E731
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # ---- timed region: device time of K steps, kernel events for the roofline
    s.profile(True)
    l0 = s.launch_count()
    _barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        t_ms = _time_steps(step, args.steps, stream, flush)
    torch.cuda.synchronize()
    _barrier(world)
    launches = s.launch_count() - l0
    dense_kind = s.dense_kernel()
    dense_ms, dense_n = s.profile_read(sd.SD_KERNEL_DENSE)
    epi_ms, _ = s.profile_read(sd.SD_KERNEL_EPILOGUE)
    near_ms, _ = s.profile_read(sd.SD_KERNEL_NEAR)
    cells_ms, _ = s.profile_read(sd.SD_KERNEL_CELLS)
    s.profile(False)
    t_ms = _max_over_ranks(t_ms, world)
    ms_step = t_ms / args.steps
    value = world * float(n) * n / (ms_step * 1e-3)

    # ---- end to end through the public API with pinned host buffers: every step
    # copies its input (the per-particle forces) in (H2D) and its result (the
    # positions) out (D2H), each as one asynchronous copy on the stream; the host
    # synchronises once and checks the last result
    fh = torch.from_numpy(F).pin_memory()
    outh = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    s.set_positions(x)
    _barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.set_forces(fh, asynchronous=True)        # H2D of the step's input
        s.step(DT, 1)
        s.get_positions(outh, asynchronous=True)   # D2H of the step's result
    torch.cuda.synchronize()
    e2e_s = _max_over_ranks(time.perf_counter() - t0, world)
    if not np.all(np.isfinite(outh.numpy())):
        raise RuntimeError("end-to-end loop produced non-finite positions")
    e2e_value = world * float(n) * n * args.steps / e2e_s

    clocks = clk.summary()
    peaks, peak_src = _peaks()
    sms = props.multi_processor_count
    fp32_peak = sms * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    dense_avg_ms = dense_ms / max(dense_n, 1)
    achieved = FLOPS_PER_PAIR * float(n) * n / (dense_avg_ms * 1e-3) / 1e12
    s.close()

    extra = {}
    if world > 1:
        extra.update(_leg_tile_sharded(args, x, F, stream, world, rank))
        extra.update(_leg_batched_sharded(args, stream, world, rank))
    if rank == 0 and not args.quick:
        extra.update(legs(args, x, F, stream, flush, workloads=(world == 1)))

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config(L, world),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": _dense_traffic(dense_kind),
                     "kernel": DENSE_NAMES[dense_kind],
                     "flops_per_launch": FLOPS_PER_PAIR * float(n) * n,
                     "flops_definition": "34 per ordered pair (i, j) of the sum, N^2 per launch, whichever "
                                         "kernel visits them",
                     "avg_launch_ms": dense_avg_ms, "launches": dense_n,
                     "peak_source": "%d SMs x %d FP32 lanes x 2 x %.0f MHz (sm_max_mhz, %s)"
                                    % (sms, FP32_LANES_PER_SM, peaks.get("sm_max_mhz", 2070.0), peak_src)},
        "kernel_ms_per_step": {"dense": dense_ms / args.steps, "near": near_ms / args.steps,
                               "epilogue": epi_ms / args.steps, "cells": cells_ms / args.steps,
                               "note": "CUDA-event ranges per kernel class; with Verlet lists the rebuild "
                                       "(cells) and the near pass run on a side stream beside the all-pairs "
                                       "kernel, and their ranges include time spent waiting for free SMs"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 24 * n, "d2h_bytes_per_step": 24 * n},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)


def _leg_tile_sharded(args, x, F, stream, world, rank):
    """One N = 65,536 system split over all ranks by tile shards (strong scaling): per
    step each rank runs its share of the all-pairs kernel, an NCCL all-gather brings
    every share to every rank, and every rank finishes the step.  Timed like the main
    leg (barrier, CUDA events, max over ranks)."""
    import torch
    import paper_1205_6333_gb300 as sd
    from paper_1205_6333_gb300.distributed import tile_sharded_steps
    n = x.shape[0]
    s = sd.System(n, prec="fp32c", stream="torch", torch_allocator=True, device=torch.cuda.current_device())
    s.set_positions(x)
    s.set_forces(F)
    import torch.distributed as dist
    via_host = dist.get_backend() != "nccl"
    tile_sharded_steps(s, DT, max(args.warmup, 3), rank, world, via_host=via_host)
    torch.cuda.synchronize()
    _barrier(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tile_sharded_steps(s, DT, args.steps, rank, world, via_host=via_host)
    e1.record(stream)
    torch.cuda.synchronize()
    _barrier(world)
    t_ms = _max_over_ranks(e0.elapsed_time(e1), world)
    kind = s.dense_kernel()
    s.close()
    ms = t_ms / args.steps
    return {"tile_sharded": {"value": float(n) * n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                             "scaling": "strong", "ranks": world, "n": n, "all_pairs_kernel": kind,
                             "exchange": "%s all-gather of 24 B per particle and rank per step"
                                         % ("host-staged gloo" if via_host else "NCCL")}}


def _leg_batched_sharded(args, stream, world, rank):
    """The batched workload (16,384 clusters) split over the ranks by cluster shards
    balanced by pair work; no data moves between ranks.  Steps/s of the whole batch
    from the slowest rank (strong scaling)."""
    import torch
    from paper_1205_6333_gb300 import inputs
    from paper_1205_6333_gb300.distributed import ShardedBatch
    w = inputs.config_inputs(4)
    off = w["offsets"]
    sb = ShardedBatch(off, rank, world, prec="fp32c", stream="torch", torch_allocator=True)
    sb.set_positions(w["x"])
    sb.set_forces(w["F"])
    sb.step(0.01, 16)   # (autotune, graph capture)
    torch.cuda.synchronize()
    _barrier(world)
    k = max(args.steps, 32)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sb.step(0.01, k)
    e1.record(stream)
    torch.cuda.synchronize()
    _barrier(world)
    ms = _max_over_ranks(e0.elapsed_time(e1) / k, world)
    sb.close()
    return {"batched_sharded": {"steps_per_s": 1e3 / ms, "ms_per_step": ms, "scaling": "strong", "ranks": world,
                                "clusters_this_rank_0": None if rank else sb.c1 - sb.c0,
                                "split": "contiguous clusters balanced by the sum of N_c^2, no exchange"}}


def run_leg(args):
    """One extra leg alone (used for profiling it): prints its JSON object."""
    import torch
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    x, F, _ = _main_inputs(N_MAIN)
    print(json.dumps(legs(args, x, F, stream, flush, only=args.leg)), flush=True)


def legs(args, x, F, stream, flush, only=None, workloads=True):
    """FP64 path, batched workload, Oseen variant and the CPU oracle baseline (rank 0
    only); with `workloads` (single-GPU runs) also the four-sphere runs of workload 1,
    the trajectory drift of workload 3, the adjoint of workload 5, the N sweep
    2^10 .. 2^18, the paper's fcc benchmark and the lubrication lattice."""
    out = {}
    if only in (None, "fp64"):
        out.update(_leg_fp64(args, x, F, stream, flush))
    if only in (None, "batched"):
        out.update(_leg_batched(args, stream, flush))
    if only in (None, "oseen"):
        out.update(_leg_oseen(args, x, F, stream, flush))
    if only is None and workloads:
        out.update(leg_workload1(args))
        out.update(leg_drift(args))
        out.update(leg_adjoint(args))
        out.update(leg_sweep(args, forced=False))
        out.update(leg_fcc(args))
        out.update(leg_lubrication(args))
    if only is None:
        out["cpu_baseline"] = cpu_baseline(x, F, target_s=args.cpu_seconds)
    return out


def _leg_fp64(args, x, F, stream, flush):
    import torch
    import paper_1205_6333_gb300 as sd
    n = x.shape[0]
    s = sd.System(n, prec="fp64", stream="torch")
    s.set_positions(x)
    s.set_forces(F)
    s.step(DT, 1)
    torch.cuda.synchronize()
    k = max(2, min(5, args.steps))
    t = _time_steps(lambda: s.step(DT, 1), k, stream, flush)
    s.close()
    fp64_ms = t / k
    return {"fp64": {"value": float(n) * n / (fp64_ms * 1e-3), "unit": UNIT, "ms_per_step": fp64_ms, "steps": k}}


def _dense_ms(s, k, stream, flush, step):
    """Mean event time of the all-pairs kernel over k steps (profiler on)."""
    import paper_1205_6333_gb300 as sd
    s.profile(True)
    _time_steps(step, k, stream, flush)
    ms, cnt = s.profile_read(sd.SD_KERNEL_DENSE)
    s.profile(False)
    return ms / max(cnt, 1)


def _leg_oseen(args, x, F, stream, flush):
    """The paper's Oseen-only variant (Sec. 3.3: 13% faster than Rotne-Prager on C2050)."""
    import paper_1205_6333_gb300 as sd
    n = x.shape[0]
    out = {}
    for tensor in ("rpy", "oseen"):
        s = sd.System(n, tensor=tensor, stream="torch", torch_allocator=True)
        s.set_positions(x)
        s.set_forces(F)
        s.step(DT, 3)
        out[tensor] = _dense_ms(s, max(5, min(args.steps, 20)), stream, flush, lambda: s.step(DT, 1))
        s.close()
    return {"oseen": {"dense_ms_rpy": out["rpy"], "dense_ms_oseen": out["oseen"],
                      "oseen_speedup": out["rpy"] / out["oseen"],
                      "flops_per_pair": {"rpy": 34, "oseen": 30}}}


def leg_sweep(args, forced=True):
    """N = 2^10 .. 2^18 at phi = 0.05: FP32C and FP64 step times, the all-pairs kernel's
    fraction of the FP32 peak, and the FP32C / FP64 velocity error against the oracle
    on sampled rows; with `forced`, also both all-pairs kernels forced in turn."""
    import torch
    import oracle
    import paper_1205_6333_gb300 as sd
    from paper_1205_6333_gb300 import inputs
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sms * FP32_LANES_PER_SM * 2 * _peaks()[0].get("sm_max_mhz", 2070.0) * 1e6
    rows_out = []
    for e in range(10, 19):
        n = 1 << e
        x, L = inputs.cube_rsa(n, PHI, inputs.SEED_BASE + 2)
        F = inputs.normal_forces(n, inputs.SEED_BASE + 1002)
        x = x.astype(np.float32).astype(np.float64)
        F = F.astype(np.float32).astype(np.float64)
        rows = np.random.default_rng(e).choice(n, min(n, 256), replace=False).astype(np.int32)
        ref = oracle.mobility_rows(x, F, rows, "rpy", nthreads=os.cpu_count())
        rec = {"n": n, "box_side": L}
        for prec in ("fp32c", "fp64"):
            s = sd.System(n, prec=prec, stream="torch", torch_allocator=True)
            s.set_positions(x)
            v = s.mobility_apply(F)
            den = np.linalg.norm(ref, axis=1).max()
            rec["err_" + prec] = float(np.linalg.norm(v[rows] - ref, axis=1).max() / den)
            s.set_forces(F)
            s.step(DT, 2)
            k = 10 if prec == "fp32c" else (3 if n <= 65536 else 2)
            t = _time_steps(lambda: s.step(DT, 1), k, stream, flush) / k
            rec["step_ms_" + prec] = t
            rec["pairs_per_s_" + prec] = float(n) * n / (t * 1e-3)
            if prec == "fp32c":
                dms = _dense_ms(s, 5, stream, flush, lambda: s.step(DT, 1))
                rec["dense_kernel"] = s.dense_kernel()
                rec["dense_ms"] = dms
                rec["frac_fp32_peak"] = FLOPS_PER_PAIR * float(n) * n / (dms * 1e-3) / peak
            s.close()
        # both all-pairs kernels forced, for the automatic choice between them
        for dense in (("directed", "symmetric") if forced else ()):
            s = sd.System(n, prec="fp32c", stream="torch", torch_allocator=True, dense=dense)
            s.set_positions(x)
            s.set_forces(F)
            s.step(DT, 2)
            rec["step_ms_" + dense] = _time_steps(lambda: s.step(DT, 1), 10, stream, flush) / 10
            rec["dense_ms_" + dense] = _dense_ms(s, 5, stream, flush, lambda: s.step(DT, 1))
            s.close()
        rec["fp64_over_fp32c_time"] = rec["step_ms_fp64"] / rec["step_ms_fp32c"]
        rows_out.append(rec)
        print(json.dumps(rec), file=sys.stderr, flush=True)
    return {"sweep": rows_out}


def leg_workload1(args):
    """Config 1 (Sec. 4): four spheres on a horizontal square of side 4a (+-0.01a
    seeded jitter), F = (0, 0, -1), RPY, 20,000 Euler steps at dt = 0.01 tau_s: the
    FP64 and FP32C GPU paths against the FP64 oracle, and steps/s.  Then the paper's
    symmetric start (RP tensor) for 1,000 tau_s: the orbit's period and amplitude
    (from the maxima of particle 1's x) and the drift of particles 1 and 3 out of the
    xz plane."""
    import torch
    import oracle
    import paper_1205_6333_gb300 as sd
    from paper_1205_6333_gb300 import inputs
    x0 = inputs.config_inputs(1)["x"]
    tau = 1.0 / oracle.mu0()
    dt = 0.01 * tau
    nsteps = 20000
    t0 = time.perf_counter()
    ref = oracle.euler(x0, nsteps, dt, gravity=(0, 0, -1.0))
    out = {"n": 4, "steps": nsteps, "dt_tau_s": 0.01, "oracle_s": time.perf_counter() - t0}
    disp = float(np.abs(ref - x0).max())
    for prec in ("fp64", "fp32c"):
        with sd.System(4, prec=prec, gravity=(0, 0, -1.0), stream="torch") as s:
            s.set_positions(x0)
            s.step(dt, 16)
            s.set_positions(x0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.step(dt, nsteps)
            xt = s.get_positions()
            el = time.perf_counter() - t0
        d = float(np.abs(xt - ref).max())
        out[prec] = {"max_abs_diff": d, "rel_to_max_displacement": d / disp, "steps_per_s": nsteps / el}
    with open(os.path.join(ROOT, "tests", "golden", "four_sphere_orbit.json")) as f:
        g = json.load(f)
    dto = g["dt_tau_s"] * tau
    chunk = 100
    for prec in ("fp64", "fp32c"):
        traj = []
        with sd.System(4, prec=prec, tensor="rp", gravity=g["force"], stream="torch") as s:
            s.set_positions(np.array(g["start"]))
            for _ in range(int(1000.0 / g["dt_tau_s"]) // chunk):
                s.step(dto, chunk)
                traj.append(s.get_positions())
        traj = np.array(traj)
        x1 = traj[:, 0, 0]
        k = np.nonzero((x1[1:-1] > x1[:-2]) & (x1[1:-1] >= x1[2:]))[0] + 1
        t = (k + 1) * chunk * g["dt_tau_s"]
        out["orbit_" + prec] = {
            "period_tau_s": float(np.mean(np.diff(t))) if len(t) > 1 else None,
            "paper_period_tau_s": g["period_tau_s"],
            "amplitude_x1": float(0.5 * (x1.max() - x1.min())),
            "y_drift_particles_1_3": float(np.abs(traj[:, [0, 2], 1]).max()),
            "time_tau_s": 1000.0}
    return {"workload1": out}


def leg_drift(args):
    """Workload 3: N = 16,384, phi = 0.10, gravity + eps (2a/r)^12 repulsion cut at
    2.5a, Euler dt = 1e-3.  FP32C trajectory drift against the FP64 GPU path at 10^2,
    10^3, 10^4 steps, oracle parity of both at 10^2 steps, FP32C and FP64 steps/s.
    The oracle's 100 steps run on the host cores (one left free to drive the GPU) in
    a thread beside the GPU trajectories."""
    import threading

    import torch
    import oracle
    import paper_1205_6333_gb300 as sd
    from paper_1205_6333_gb300 import inputs
    w = inputs.config_inputs(3)
    x0 = w["x"]
    n = x0.shape[0]
    cores = os.cpu_count() or 1
    ref_box = {}

    def run_oracle():
        t = time.perf_counter()
        ref_box["x"] = oracle.euler(x0, 100, 1e-3, gravity=(0.0, 0.0, -1.0), rep_eps=1.0, rep_rc=2.5,
                                    nthreads=max(1, cores - 1))
        ref_box["s"] = time.perf_counter() - t

    th = threading.Thread(target=run_oracle)
    th.start()
    kw = dict(gravity=(0.0, 0.0, -1.0), rep_eps=1.0, rep_rc=2.5, stream="torch", torch_allocator=True)
    s32 = sd.System(n, prec="fp32c", **kw)
    s64 = sd.System(n, prec="fp64", **kw)
    for s in (s32, s64):
        s.set_positions(x0)
    out = {"n": n, "dt": 1e-3, "checkpoints": [], "fp64_kernel": s64.dense_kernel()}
    done = 0
    t32 = t64 = 0.0
    snaps = {}
    for target in (100, 1000, 10000):
        for sys_, key in ((s32, "32"), (s64, "64")):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            sys_.step(1e-3, target - done)
            e1.record()
            torch.cuda.synchronize()
            if key == "32":
                t32 += e0.elapsed_time(e1)
            else:
                t64 += e0.elapsed_time(e1)
        done = target
        a, b = s32.get_positions(), s64.get_positions()
        snaps[target] = (a, b)
        disp = np.abs(b - x0).max()
        rec = {"step": target, "max_abs_diff": float(np.abs(a - b).max()),
               "rel_to_max_displacement": float(np.abs(a - b).max() / disp), "max_displacement": float(disp)}
        out["checkpoints"].append(rec)
        print(json.dumps(rec), file=sys.stderr, flush=True)
    th.join()
    a, b = snaps[100]
    ref = ref_box["x"]
    dref = np.abs(ref - x0).max()
    out["checkpoints"][0]["oracle_rel_err_fp32c"] = float(np.abs(a - ref).max() / dref)
    out["checkpoints"][0]["oracle_rel_err_fp64"] = float(np.abs(b - ref).max() / dref)
    out["oracle_100_steps_s"] = ref_box["s"]
    out["fp32c_steps_per_s"] = 1e3 * done / t32
    out["fp64_steps_per_s"] = 1e3 * done / t64
    s32.close()
    s64.close()
    return {"drift": out}


def leg_lubrication(args):
    """Lubrication (Sec. 2.3, lagged velocities of Sec. 3.1): N = 32^3 = 32,768 spheres on
    a jittered simple-cubic lattice of spacing 2.9a (phi = 0.17, every nearest-neighbour
    gap inside the friction window), forces N(0,1), dt = 0.02, 40 steps (the lagged
    friction is stable there; under gravity the cluster's collective shear closes gaps
    until it is not).  FP32C steps/s with and without the friction, the FP64
    neighbour-pass time per step, and the FP32C-vs-FP64 trajectory difference."""
    import torch
    import paper_1205_6333_gb300 as sd
    from paper_1205_6333_gb300 import inputs
    m, spacing, steps = 32, 2.9, 40
    rng = np.random.default_rng(inputs.SEED_BASE + 70)
    g = np.arange(m) * spacing
    x0 = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    x0 = x0 + rng.uniform(-0.05, 0.05, x0.shape)
    n = x0.shape[0]
    fe = inputs.normal_forces(n, inputs.SEED_BASE + 71)
    stream = torch.cuda.current_stream()
    out = {"n": n, "lattice_spacing_a": spacing, "dt": 0.02}
    pos = {}
    for lub in (False, True):
        for prec in ("fp32c", "fp64"):
            s = sd.System(n, prec=prec, lubrication=lub, stream="torch", torch_allocator=True)
            s.set_positions(x0)
            s.set_forces(fe)
            if prec == "fp32c":
                s.step(0.02, 3)
                s.set_positions(x0)
                s.profile(True)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.step(0.02, steps)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / steps
                fms, fcnt = s.profile_read(sd.SD_KERNEL_FORCES)
                s.profile(False)
                key = "lub" if lub else "plain"
                out["steps_per_s_" + key] = 1e3 / ms
                out["forces_ms_per_step_" + key] = fms / steps
            else:
                s.step(0.02, steps)
            pos[(lub, prec)] = s.get_positions()
            s.close()
    a, b = pos[(True, "fp32c")], pos[(True, "fp64")]
    disp = np.linalg.norm(b - x0, axis=1).max()
    out["steps"] = steps
    out["fp32c_vs_fp64_rel_to_displacement"] = float(np.linalg.norm(a - b, axis=1).max() / disp)
    out["lub_effect_rel_to_displacement"] = float(np.linalg.norm(pos[(False, "fp64")] - b, axis=1).max() / disp)
    print(json.dumps(out), file=sys.stderr, flush=True)
    return {"lubrication": out}


def leg_fcc(args):
    """The paper's runtime benchmark (Sec. 3.3): a sedimenting fcc lattice at number
    density 0.1/a^3 in a periodic cube (nearest image only), the same force (0, 0, -1) on
    every sphere, Euler dt = 0.001 tau_s, 100 steps; N = 4 m^3 from 108 to 202,612.
    Device time per step (CUDA events around the 100 steps, replayed from the captured
    graphs) in FP32C with and without lubrication, and in FP64 up to N = 32,000; the N
    where the time per step turns from flat (launch- and latency-bound) to quadratic."""
    import torch
    import paper_1205_6333_gb300 as sd
    from paper_1205_6333_gb300 import inputs
    stream = torch.cuda.current_stream()
    tau_s = 6.0 * math.pi            # a / (mu0 F) with a = eta = F = 1
    dt = 0.001 * tau_s
    rows = []

    def time_steps(s, x, k):
        s.step(dt, 16)               # warm-up, graphs captured
        s.set_positions(x)           # fresh start (with lubrication: no previous velocities)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(dt, k)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    for m in (3, 4, 5, 6, 8, 10, 13, 16, 20, 25, 32, 37):
        x, L = inputs.fcc_lattice(m)
        n = x.shape[0]
        rec = {"n": n, "box_side": L}
        # With lubrication only 5 steps: on this lattice (gap s = 0.42, 12 neighbours) the
        # lagged friction has spectral radius mu zeta > 1, so rounding noise in the
        # relative velocities grows ~3x per step; 5 steps stay at rounding level.
        for key, prec, lub, k in (("fp32c", "fp32c", False, 100), ("fp32c_lub", "fp32c", True, 5),
                                  ("fp64", "fp64", False, 10 if n > 8192 else 100)):
            if prec == "fp64" and n > 32000:
                continue
            s = sd.System(n, prec=prec, gravity=(0.0, 0.0, -1.0), box=(L, L, L), lubrication=lub,
                          stream="torch", torch_allocator=True)
            s.set_positions(x)
            rec["ms_per_step_" + key] = time_steps(s, x, k)
            xT = s.get_positions()
            d = xT - x
            # uniform sedimentation of a perfect periodic lattice: every sphere moves alike
            rec["spread_" + key] = float(np.abs(d - d.mean(axis=0)).max() / max(np.abs(d).max(), 1e-300))
            if key == "fp32c":
                rec["dense_kernel"] = s.dense_kernel()
            s.close()
        rec["pairs_per_s_fp32c"] = float(n) * n / (rec["ms_per_step_fp32c"] * 1e-3)
        rows.append(rec)
        print(json.dumps(rec), file=sys.stderr, flush=True)
    # crossover: t(N) = t0 + c N^2 with t0 the small-N floor and c from the largest N
    t0 = min(r["ms_per_step_fp32c"] for r in rows)
    big = rows[-1]
    c = (big["ms_per_step_fp32c"] - t0) / float(big["n"]) ** 2
    out = {"rows": rows, "flat_ms_per_step": t0, "ms_per_pair_large_n": c,
           "crossover_n": math.sqrt(t0 / c),
           "paper_context": "Tesla C2050: linear in N up to about 2,000 particles, quadratic above; 5.7 ms per "
                            "step at N = 4,150 with lubrication (Sec. 3.3)"}
    return {"fcc": out}


def leg_access(args, sizes=(70000, 262144), reps=10):
    """The memory-access study of App. A: the naive, tiling and small-tiling kernels
    (plus tiles copied by cp.async.bulk for the linear map) under the linear, strided
    and unordered maps, float and float4, 128 threads per block as in the study.
    Device time per launch (CUDA events, 3 warm-up and `reps` timed launches) divided
    by N^2; N = 70,000 is the top of the study's range, 262,144 a larger array (4 MB as
    float4).  Both arrays fit in L2: the study measures what the caches and shared
    memory do with each access pattern, so there is no L2 flush.  Inputs are small
    integers, so every sum is exact and each launch is checked against the closed form
    of the linear map (in[j] + sum(in), the same for the strided and unordered naive
    kernels at N coprime to 131)."""
    import torch
    import paper_1205_6333_gb300 as sd
    stream = torch.cuda.current_stream()
    rows = []
    for n in sizes:
        for vec4 in (False, True):
            g = torch.Generator().manual_seed(n + vec4)
            shape = (n, 4) if vec4 else (n,)
            x = torch.randint(-8, 9, shape, generator=g).to(torch.float32).cuda()
            closed = (x + x.sum(dim=0)).cpu().numpy()   # exact: |sums| < 2^24
            out = torch.empty_like(x)
            for algo in ("naive", "tiling", "smalltiling", "bulk"):
                for kind in ("linear", "strided", "unordered"):
                    if algo == "bulk" and kind != "linear":
                        continue
                    for _ in range(3):
                        sd.access_study(algo, kind, x, block=128, out=out)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    for _ in range(reps):
                        sd.access_study(algo, kind, x, block=128, out=out)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    sd.sd_access_status()
                    ms = e0.elapsed_time(e1) / reps
                    rec = {"n": n, "type": "float4" if vec4 else "float", "algo": algo, "map": kind,
                           "ms": ms, "ps_per_pair": ms * 1e9 / (float(n) * n),
                           "loaded_gbs": float(n) * n * (16 if vec4 else 4) / (ms * 1e-3) / 1e9}
                    if algo == "naive" or kind != "unordered":
                        rec["exact"] = bool(np.array_equal(out.cpu().numpy(), closed))
                    rows.append(rec)
                    print(json.dumps(rec), file=sys.stderr, flush=True)
    return {"access": {"rows": rows, "block": 128, "reps": reps,
                       "paper_context": "Tesla T10 / C2050 (App. A): time per N^2 converged by N = 70,000; "
                                        "on the cached C2050 the naive kernel is as fast as tiling for the "
                                        "linear and strided maps"}}


def leg_adjoint(args, n_fd=16):
    """Workload 5: N = 4,096, phi = 0.05, gravity, dt = 0.01, 1000 Euler steps,
    L = sum |x_i(T) - x_i*|^2, checkpoints every 50 steps.  Central finite differences
    (h = 1e-4) of the FP64 GPU path on n_fd seeded components of x0 and of F, the
    FP32C-forward gradient against the FP64 one, and the backward/forward time ratio."""
    import torch
    import paper_1205_6333_gb300 as sd
    from paper_1205_6333_gb300 import inputs
    w = inputs.config_inputs(5)
    x0, target = w["x"], w["target"]
    n = x0.shape[0]
    nsteps, dt, K, h = 1000, 0.01, 50, 1e-4
    fe = np.zeros_like(x0)
    res = {}
    grads = {}
    for prec in ("fp64", "fp32c"):
        s = sd.System(n, prec=prec, gravity=(0.0, 0.0, -1.0), stream="torch", torch_allocator=True)
        s.set_positions(x0)
        s.set_forces(fe)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(dt, nsteps)
        xT = s.get_positions()
        tf = time.perf_counter() - t0
        s.set_positions(x0)
        t0 = time.perf_counter()
        gx0, gF = s.adjoint(dt, nsteps, K, 2.0 * (xT - target))
        tb = time.perf_counter() - t0
        grads[prec] = (gx0, gF)
        res[prec] = {"forward_s": tf, "backward_s": tb, "backward_over_forward": tb / tf}
        if prec == "fp64":
            def loss(x, f):
                s.set_positions(x)
                s.set_forces(f)
                s.step(dt, nsteps)
                return float(((s.get_positions() - target) ** 2).sum())
            rng = np.random.default_rng(inputs.SEED_BASE + 55)
            errs_x, errs_f = [], []
            for comp in rng.choice(3 * n, n_fd, replace=False):
                i, d = divmod(int(comp), 3)
                e = np.zeros_like(x0)
                e[i, d] = h
                fdx = (loss(x0 + e, fe) - loss(x0 - e, fe)) / (2 * h)
                fdf = (loss(x0, fe + e) - loss(x0, fe - e)) / (2 * h)
                # relative to the component, floored at 1e-3 of the gradient's scale
                errs_x.append(abs(gx0[i, d] - fdx) / max(abs(fdx), 1e-3 * np.abs(gx0).max()))
                errs_f.append(abs(gF[i, d] - fdf) / max(abs(fdf), 1e-3 * np.abs(gF).max()))
            res["fd_components"] = n_fd
            res["fd_max_rel_err_x0"] = float(max(errs_x))
            res["fd_max_rel_err_F"] = float(max(errs_f))
        s.close()
    for k, nm in ((0, "x0"), (1, "F")):
        a, b = grads["fp32c"][k], grads["fp64"][k]
        res["fp32c_vs_fp64_rel_err_" + nm] = float(np.abs(a - b).max() / np.abs(b).max())
    return {"adjoint": res}


def _leg_batched(args, stream, flush):
    """Batched clusters (16,384 clusters, N ~ U{4..256}, phi = 0.05, forces N(0,1))."""
    import torch
    import paper_1205_6333_gb300 as sd
    from paper_1205_6333_gb300 import inputs
    w = inputs.config_inputs(4)
    off = w["offsets"]
    sizes = np.diff(off).astype(np.int64)
    pairs = float((sizes ** 2).sum())
    b = sd.Batch(off, prec="fp32c", stream="torch", torch_allocator=True)
    b.set_positions(w["x"])
    b.set_forces(w["F"])
    shapes = b.shapes()
    if args.batched_shape == "auto":
        choice = b.autotune()
    else:   # pinned: the most resident CTAs of the symmetric kernel, or of the one-target block kernel
        r = 0 if args.batched_shape == "sym" else 1
        choice = max(k for k, sh in enumerate(shapes) if sh["targets_per_thread"] == r and sh["threads"] == 128)
        b.set_shape(choice)
    b.step(0.01, 3)
    torch.cuda.synchronize()
    kb = max(args.steps, 10)
    b.profile(True)
    tb = _time_steps(lambda: b.step(0.01, 1), kb, stream, flush)
    bk_ms, bk_n = b.profile_read(sd.SD_KERNEL_BATCHED)
    b.profile(False)
    # steady state through the captured graph (16 steps per replay)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(0.01, 160)
    e1.record(stream)
    torch.cuda.synchronize()
    g_ms = e0.elapsed_time(e1) / 160
    # the workload's whole protocol: 1000 steps from the initial state (overlaps develop)
    b.set_positions(w["x"])
    torch.cuda.synchronize()
    e0.record(stream)
    b.step(0.01, 1000)
    e1.record(stream)
    torch.cuda.synchronize()
    p_ms = e0.elapsed_time(e1) / 1000
    b.close()
    P = int(off[-1])
    bytes_step = P * (24 + 16 + 24)
    ms_b = tb / kb
    return {"batched": {
        "steps_per_s": 1e3 / ms_b, "ms_per_step": ms_b, "graph_ms_per_step": g_ms,
        "protocol_1000_steps_ms_per_step": p_ms, "protocol_1000_steps_per_s": 1e3 / p_ms,
        "graph_steps_per_s": 1e3 / g_ms, "pairs_per_s": pairs / (ms_b * 1e-3),
        "clusters": int(len(sizes)), "particles": P, "pairs_per_step": pairs,
        "kernel_avg_ms": bk_ms / max(bk_n, 1),
        "kernel_tflops": FLOPS_PER_PAIR * pairs / (bk_ms / max(bk_n, 1) * 1e-3) / 1e12,
        "algorithmic_gbs": bytes_step / (bk_ms / max(bk_n, 1) * 1e-3) / 1e9,
        "autotune_choice": int(choice), "shape": shapes[choice], "steps": kb}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="main leg only")
    ap.add_argument("--leg", default="all", choices=["all", "main", "fp64", "batched", "oseen", "sweep", "drift",
                                                     "adjoint", "lubrication", "fcc", "access", "workload1"],
                    help="run one leg alone and print its numbers (profiling)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--batched-shape", default="auto", choices=["auto", "sym", "blocks"],
                    help="batched leg: the autotuner's shape, or the symmetric / block kernel pinned (profiling)")
    ap.add_argument("--dense", default="auto", choices=["auto", "directed", "symmetric"],
                    help="all-pairs kernel of the main leg (auto: the library's choice, symmetric at this N)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.leg in ("fp64", "batched", "oseen"):
        run_leg(args)
    elif args.leg == "sweep":
        print(json.dumps(leg_sweep(args)), flush=True)
    elif args.leg == "drift":
        print(json.dumps(leg_drift(args)), flush=True)
    elif args.leg == "adjoint":
        print(json.dumps(leg_adjoint(args)), flush=True)
    elif args.leg == "lubrication":
        print(json.dumps(leg_lubrication(args)), flush=True)
    elif args.leg == "fcc":
        print(json.dumps(leg_fcc(args)), flush=True)
    elif args.leg == "access":
        print(json.dumps(leg_access(args)), flush=True)
    elif args.leg == "workload1":
        print(json.dumps(leg_workload1(args)), flush=True)
    else:
        if args.leg == "main":
            args.quick = True
        run_ours(args)


if __name__ == "__main__":
    main()
