#!/usr/bin/env python3
"""Benchmark of the hot path: one full Algorithm 1 fit (steps A1-A6) on the
2000 x 2000 planted-sparse-line workload, through the C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints ONE JSON line (rank 0).  A step is one fit of a fresh-in-HBM, seeded
2000 x 2000 float32 matrix (lambda = 0.5): ratio staging, every (jhat, k)
weighted median, residuals, per-jhat objectives and the argmin.  The metric is
(jhat, k) weighted-median pairs per second (m (m - 1) pairs per fit); fits/s
rides along.  L2 is flushed (a 512 MiB write) before every timed step.

Under torchrun each rank fits its own seeded instance on its own GPU (weak
scaling, no collective on the data path); the job's value is all ranks' pairs
divided by the slowest rank's time.  The line then also carries `sharded`: one
fit split over all ranks by jhat (strong scaling); --sharded makes that the
headline.

Context lines beside the headline (not in `value`): the float64 fit, the
lambda batch, Algorithm 2 over every pair (with its HBM and issue ceilings),
Algorithms 2 + 3 at 1000 x 500 and 2000 x 2000, the uneven batch, the small
fit, the learned proposer, the comparison data and successive components.

--impl reference times the CPU oracle (C, OpenMP over jhat) on the machine's host
cores, on a bounded sample of the same workload (a subset of the jhat columns,
all k), in the same unit.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_ROWS, N_COLS, LAMBDA = 2000, 2000, 0.5
METRIC = "(jhat,k) weighted-median pairs/s (full m^2 scan, Algorithm 1 fit)"
UNIT = "pairs/s"
WORKLOAD = ("planted sparse line, n=2000 points x m=2000 coords, float32, 20-sparse unit-l1 "
            "v*, Laplace(0,0.1) noise, 5% N(0,100 I) outlier rows, lambda=0.5, full m^2 scan")
# Algorithmic issue count per (pair, row) element: load x_ik, ratio (one
# multiply by a per-column reciprocal), key, one pivot compare + weight add,
# residual fma + abs-add.  The ALU roofline divides by the SM issue rate.
ALG_INSTR_PER_ELEM = 8
SMS, LANES_PER_SM_CLK, SM_MAX_MHZ = 152, 128, 2070.0
# Algorithmic bytes per (jhat, k) pair of the float32 pair kernel for its
# memory ceilings: shared memory -- 16 bytes per row, a 4-byte key and a 4-byte
# weight written once and read once (the kernel itself reads 12 staged bytes
# per row: reciprocal, 32-bit weight and value); L2 -- column k read once and
# column jhat once per CTA of T_k pairs, 4 n (1 + 1/T_k) bytes.
# The peaks are measured in the same run by the library's bandwidth probes.
SMEM_BYTES_PER_ROW = 16


def _env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def job_ms(local_ms: float, dist=None, device=None) -> float:
    """The job's time over ranks: the slowest rank's (all-reduce MAX); the
    local time without a process group."""
    if dist is None:
        return local_ms
    import torch
    t = torch.tensor([local_ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, steps: int, units_per_step: float, tot_ms: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * steps * units_per_step / (tot_ms * 1e-3)


def sharded_summary(world: int, steps: int, pairs: int, step_ms, identical) -> dict:
    """The line of one fit split over `world` ranks by jhat (strong scaling):
    `step_ms` are the slowest rank's per-step times; every step is ONE fit, so
    the job's value is one fit's pairs per step time, whatever the world size."""
    tot = sum(step_ms)
    return {"workload": "one 2000 x 2000 float32 fit split over the ranks by jhat "
                        "(contiguous jhat ranges, fit_subset on each rank; the argmin over "
                        "jhat is the one exchange: three small all-reduces per fit)",
            "scaling": "strong", "n_gpus": world, "steps": steps,
            "ms_per_step": tot / steps, "value": steps * pairs / (tot * 1e-3), "unit": UNIT,
            "fits_per_s": steps / (tot * 1e-3), "identical_to_one_gpu": identical}


def measure_sharded(dev, stream, dist, steps, warmup, flush=None):
    """One fit of the seed-0 2000 x 2000 matrix split over this job's ranks
    (sharded.fit_sharded: every rank holds the same matrix and scores its own
    jhat range; NCCL all-reduces pick the argmin).  Each step is timed with
    CUDA events on the launching stream (the collectives follow it there),
    L2 flushed first; the per-step times are max-reduced over ranks.  Rank 0
    also checks the result against its own one-GPU fit, bit for bit."""
    import numpy as np
    import torch

    from paper_2402_16712_gb300 import datagen, l1line, sharded
    X, lams, _ = datagen.paper_size("float32", seed=0)
    n, m = X.shape
    Xd = torch.from_numpy(X).to(dev)
    ws = l1line.Workspace.for_shape(torch.float32, n, m, 1, dev)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            out = sharded.fit_sharded(Xd, lams, workspace=ws, stream=stream)
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    if dist is not None:
        dist.barrier()
    with torch.cuda.stream(stream):
        for a, b in ev:
            if flush is not None:
                flush.fill_(7)
            a.record(stream)
            out = sharded.fit_sharded(Xd, lams, workspace=ws, stream=stream)
            b.record(stream)
    torch.cuda.synchronize(dev)
    ms = [job_ms(a.elapsed_time(b), dist, dev) for a, b in ev]
    identical = None
    if dist is None or dist.get_rank() == 0:
        v1, o1, j1, _ = l1line.fit(Xd, lams, workspace=ws, stream=stream)
        if stream is not None:
            stream.synchronize()
        vs, os_, js = (t.cpu().numpy() for t in out)
        identical = bool(np.array_equal(v1.cpu().numpy().view(np.uint32), vs.view(np.uint32))
                         and np.array_equal(o1.cpu().numpy().view(np.int64), os_.view(np.int64))
                         and np.array_equal(j1.cpu().numpy(), js))
    world = dist.get_world_size() if dist is not None else 1
    return sharded_summary(world, steps, m * (m - 1), ms, identical)


def _src_hash() -> str:
    """Hash of the pair kernel's code (comments and whitespace stripped, so a
    comment edit does not orphan the committed ncu summaries)."""
    h = hashlib.sha256()
    for f in ("k_pairs.cu", "k_pairs_shape.cu", "pairs.cuh", "select32.cuh", "common.cuh",
              "binmap.cuh"):
        src = open(os.path.join(ROOT, "paper_2402_16712_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def _profile_traffic():
    """DRAM bytes per pair-kernel launch from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "launches_paper_size_f32.md")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m_hash = re.search(r"source_hash:\s*([0-9a-f]+)", txt)
    m_bytes = re.search(r"dram_bytes_per_launch_full:\s*([0-9.eE+]+)", txt)
    if not m_hash or not m_bytes or m_hash.group(1) != _src_hash():
        return None
    return float(m_bytes.group(1))


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = f"/tmp/l1line_clocks_{os.getpid()}.csv"

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "samples": len(sm), "reasons": sorted(reasons)}


def _host_cores() -> int:
    """Host cores this process may run on.  Not OpenMP's default team size:
    torchrun sets OMP_NUM_THREADS=1 for every rank, while the oracle timings
    run on rank 0 alone and use all the cores."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_baseline(X, lam, target_s=12.0):
    """The oracle as it stands on the host cores, on a bounded sample: the first
    J jhat columns (all k), J grown until the run takes a few seconds."""
    import oracle
    nth = _host_cores()
    J = max(1, nth)
    while True:
        t0 = time.perf_counter()
        oracle.fit(X, [lam], jlist=list(range(J)), nthreads=nth, want_all=False)
        dt = time.perf_counter() - t0
        if dt >= target_s / 4 or J >= X.shape[1]:
            break
        J = min(X.shape[1], int(J * max(2.0, target_s / 4 / max(dt, 1e-3))))
    m = X.shape[1]
    pairs = J * (m - 1)
    # the same oracle on one core, on a sample of about the same duration
    J1 = max(1, J // nth)
    t0 = time.perf_counter()
    oracle.fit(X, [lam], jlist=list(range(J1)), nthreads=1, want_all=False)
    dt1 = time.perf_counter() - t0
    return {"value": pairs / dt, "unit": UNIT, "cores": nth, "kind": "oracle",
            "sample": f"{J} of {m} jhat columns x all {m - 1} k (one lambda), {dt:.2f} s",
            "single_core": {"value": J1 * (m - 1) / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"{J1} of {m} jhat columns x all {m - 1} k, {dt1:.2f} s"},
            "seconds": dt, "fits_per_s": (pairs / dt) / (m * (m - 1))}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    from paper_2402_16712_gb300 import datagen
    import oracle
    X, lams, _ = datagen.paper_size("float32")
    lam = float(lams[0])
    nth = _host_cores()
    m = X.shape[1]
    # each step: a sample of jhat columns sized to a couple of seconds
    J = nth
    t0 = time.perf_counter()
    oracle.fit(X, [lam], jlist=list(range(J)), nthreads=nth, want_all=False)
    dt = time.perf_counter() - t0
    J = max(1, min(m, int(J * 2.0 / max(dt, 1e-3))))
    for _ in range(args.warmup):
        oracle.fit(X, [lam], jlist=list(range(J)), nthreads=nth, want_all=False)
    times = []
    for s in range(args.steps):
        cols = [(s * J + q) % m for q in range(J)]
        t0 = time.perf_counter()
        oracle.fit(X, [lam], jlist=cols, nthreads=nth, want_all=False)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.steps * J * (m - 1) / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_ROWS, "m": N_COLS, "lambda": LAMBDA,
                   "parallelism": "host cores (OpenMP over jhat)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nth, "kind": "oracle",
                         "sample": f"each step: {J} of {m} jhat columns x all k"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2402_16712_gb300 import autotune, datagen, l1line

    rank, world, local = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if rank == 0 or world == 1:
        import __graft_entry__
        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
    l1line.load()

    X, lams, _ = datagen.paper_size("float32", seed=rank)
    n, m = X.shape
    pairs = m * (m - 1)
    stream = torch.cuda.Stream(device=dev)
    Xd = torch.from_numpy(X).to(dev)
    ws = l1line.Workspace.for_shape(torch.float32, n, m, 1, dev)
    out = (torch.empty((1, m), dtype=torch.float32, device=dev),
           torch.empty(1, dtype=torch.float64, device=dev),
           torch.empty(1, dtype=torch.int32, device=dev))
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for a, b in ev + kev:  # create the events
            a.record(stream)
            b.record(stream)
        for _ in range(args.warmup):
            l1line.fit(Xd, lams, workspace=ws, stream=stream, out=out)
    stream.synchronize()
    rc = l1line.status(ws, stream)
    if rc != l1line.OK:
        raise SystemExit(f"fit failed on the device: {l1line.status_string(rc)}")
    # the library's autotuner picks the pair kernel's launch for this shape
    # (untimed; results do not depend on it)
    with torch.cuda.stream(stream):
        tuning = autotune.apply(torch.float32, n, m, 1, flush=flush,
                                run=lambda: l1line.fit(Xd, lams, workspace=ws, stream=stream,
                                                       out=out))
        for _ in range(2):
            l1line.fit(Xd, lams, workspace=ws, stream=stream, out=out)
    stream.synchronize()
    launches_per_fit = l1line.last_launch_count()

    # ---- timed region: K fits, L2 flushed before each ----------------------
    clk = Clocks(dev.index)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clk.start()
    with torch.cuda.stream(stream):
        for s in range(args.steps):
            flush.fill_(s & 0xFF)
            l1line.profile_events(*kev[s])
            ev[s][0].record(stream)
            l1line.fit(Xd, lams, workspace=ws, stream=stream, out=out)
            ev[s][1].record(stream)
    l1line.profile_events()
    torch.cuda.synchronize(dev)
    clocks = clk.stop()
    if dist is not None:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    kern_ms = [a.elapsed_time(b) for a, b in kev]
    tot_ms = sum(step_ms)
    rc = l1line.status(ws, stream)
    if rc != l1line.OK:
        raise SystemExit(f"fit failed on the device: {l1line.status_string(rc)}")
    tot_ms = job_ms(tot_ms, dist, dev)
    value = job_value(world, args.steps, pairs, tot_ms)

    # ---- float64 input, same workload (reported beside the headline) -------
    l1line.set_tuning(None)
    X64 = X.astype(np.float64)
    Xd64 = torch.from_numpy(X64).to(dev)
    ws64 = l1line.Workspace.for_shape(torch.float64, n, m, 1, dev)
    with torch.cuda.stream(stream):
        for _ in range(2):
            l1line.fit(Xd64, lams, workspace=ws64, stream=stream)
        tuning64 = autotune.apply(torch.float64, n, m, 1, flush=flush,
                                  run=lambda: l1line.fit(Xd64, lams, workspace=ws64,
                                                         stream=stream))
        l1line.fit(Xd64, lams, workspace=ws64, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k64 = max(2, args.steps // 4)
        e0.record(stream)
        for _ in range(k64):
            l1line.fit(Xd64, lams, workspace=ws64, stream=stream)
        e1.record(stream)
    stream.synchronize()
    ms64 = e0.elapsed_time(e1) / k64
    plan64 = l1line.plan(torch.float64, n, m)  # the launch the double steps ran
    l1line.set_tuning(None)

    # ---- end to end through the ABI with host buffers ----------------------
    l1line.set_tuning(tuning or None)  # this rank's tuning of the timed steps
    plan = l1line.plan(torch.float32, n, m)  # the launch the timed steps ran
    Xh = torch.from_numpy(X).pin_memory()
    vh = torch.empty((1, m), dtype=torch.float32).pin_memory()
    oh = torch.empty(1, dtype=torch.float64).pin_memory()
    jh = torch.empty(1, dtype=torch.int32).pin_memory()
    e2e_steps = max(3, args.steps // 2)
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e2e_steps):
            Xd.copy_(Xh, non_blocking=True)
            l1line.fit(Xd, lams, workspace=ws, stream=stream, out=out)
            vh.copy_(out[0], non_blocking=True)
            oh.copy_(out[1], non_blocking=True)
            jh.copy_(out[2], non_blocking=True)
        e1.record(stream)
    stream.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    d2h = vh.numel() * 4 + 8 + 4

    extras = {} if args.no_extras else measure_extras(dev, stream, flush)
    if world > 1:  # one fit split over the ranks (strong scaling), beside the replicas
        extras["sharded"] = measure_sharded(dev, stream, dist, max(3, args.steps // 2), 3, flush)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    kms = statistics.mean(kern_ms)
    l2_gbs, smem_gbs = measure_ceilings(dev, stream)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "m": m, "lambda": float(lams[0]),
                   "pairs_per_fit": pairs, "parallelism": f"replicas x{world} (one instance per GPU)",
                   "l2": "flushed before every timed step (512 MiB write)",
                   "tuning": {"applied": tuning, "plan": plan}},
        "fits_per_s": world * args.steps / (tot_ms * 1e-3),
        "f64": {"ms_per_step": ms64, "value": pairs / (ms64 * 1e-3), "unit": UNIT,
                "tuning": {"applied": tuning64, "plan": plan64},
                "roofline": roofline(n, pairs, ms64, plan64["kchunk"], plan64["column"], l2_gbs,
                                     smem_gbs, None,
                                     pair_shape(plan64["warps"], plan64["ctas_per_sm"]),
                                     dtype="double", timed="whole fit")},
        "roofline": roofline(n, pairs, kms, plan["kchunk"], plan["column"], l2_gbs,
                             smem_gbs, _profile_traffic(),
                             pair_shape(plan["warps"], plan["ctas_per_sm"])),
        "e2e": {"value": pairs / (e2e_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": int(X.nbytes), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches_per_fit * args.steps,
        "clocks": clocks,
    }
    line.update(extras)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = {k: v for k, v in cpu_baseline(X, float(lams[0])).items()
                                if k in ("value", "unit", "cores", "kind", "sample",
                                         "single_core")}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def measure_ceilings(dev, stream):
    """Measured L2 and shared-memory read bandwidth (GB/s, best of a few
    probes): a 64 MB L2-resident buffer read 20 times; every SM reading its
    shared memory conflict-free."""
    import torch

    from paper_2402_16712_gb300 import l1line
    buf = torch.ones(64 << 20, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        l1line.probe_bandwidth(l1line.PROBE_L2, 2, buf, stream)
        l2 = max(l1line.probe_bandwidth(l1line.PROBE_L2, 20, buf, stream) for _ in range(5))
        l1line.probe_bandwidth(l1line.PROBE_SMEM, 16, None, stream)
        sm = max(l1line.probe_bandwidth(l1line.PROBE_SMEM, 4000, None, stream) for _ in range(3))
    return l2 / 1e9, sm / 1e9


def pair_shape(warps, ctas):
    """The library's launch shape for warps per CTA x CTAs per SM (the rule of
    pair_shape in csrc/k_pairs.cu): 2 = 128 registers (<= 16 resident warps),
    0 = 80 registers (17-24 resident, CTAs of <= 8 warps), 1 = 64 registers (25-32)."""
    t = warps * ctas
    return 2 if t <= 16 else (0 if t <= 24 else 1)


def roofline(n, pairs, kms, kchunk, column, l2_gbs, smem_gbs, traffic, shape=0,
             dtype="float", timed="pair kernel"):
    """The pair kernel against its three ceilings; the binding one (the fewest
    pairs/s) is the headline roofline.  kchunk, column and shape are those of
    the timed launch's plan (column 1: x_ijhat staged in shared memory).  The
    double fit has the same ceilings: it selects on the same 32-bit weights
    and staged arrays, and its residual runs in float-float arithmetic; kms
    is then the whole fit's time (timed says which)."""
    pps = pairs / (kms * 1e-3)
    alu_peak = SMS * LANES_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e12
    per = {
        "smem": (SMEM_BYTES_PER_ROW * n, smem_gbs * 1e9, 1e9, "GB/s",
                 f"{SMEM_BYTES_PER_ROW} shared-memory bytes per (pair,row): staged 1/x_ijhat, "
                 "q_i and x_ijhat read once each; peak = shared-memory read probe, this run"),
        "l2": (4.0 * n * (1.0 + 1.0 / max(1, kchunk)), l2_gbs * 1e9, 1e9, "GB/s",
               f"4 n (1 + 1/T_k) bytes per pair, T_k = {kchunk}; peak = L2 read probe "
               "(64 MB resident buffer), this run"),
        "alu": (ALG_INSTR_PER_ELEM * n, alu_peak * 1e12, 1e12, "Tinstr/s",
                f"{ALG_INSTR_PER_ELEM} lane-instructions per (pair,row); peak = {SMS} SMs x "
                f"{LANES_PER_SM_CLK} lanes x {SM_MAX_MHZ:.0f} MHz"),
    }
    ceilings = {}
    for name, (work, peak, scale, unit, basis) in per.items():
        ceilings[name] = {"achieved": pps * work / scale, "peak": peak / scale, "unit": unit,
                          "frac": pps * work / peak, "ceiling_pairs_per_s": peak / work,
                          "basis": basis}
    bound = min(ceilings, key=lambda c: ceilings[c]["ceiling_pairs_per_s"])
    c = ceilings[bound]
    return {"bound": bound, "achieved": c["achieved"], "peak": c["peak"], "unit": c["unit"],
            "frac": c["frac"], "traffic": traffic,
            "kernel": f"k_pairs<{dtype}, 0, {1 if column == 1 else 0}, {shape}>",
            "kernel_ms": kms, "timed": timed, "basis": c["basis"], "ceilings": ceilings}


def _replay_ms(g, stream, steps, flush=None):
    """Mean device time of `steps` replays of graph g on `stream` (events per
    replay; L2 flushed before each when `flush` is given)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    with torch.cuda.stream(stream):
        for _ in range(3):
            g.replay()
        for a, b in ev:
            if flush is not None:
                flush.fill_(1)
            a.record(stream)
            g.replay()
            b.record(stream)
    stream.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in ev)


def measure_extras(dev, stream, flush):
    """The other workloads, reported beside the headline (not in `value`):
    the lambda batch and the uneven batch (each captured once into a CUDA graph
    and replayed), Algorithm 2 over every pair of the 2000 x 2000 matrix (with
    its HBM and issue ceilings), Algorithms 2 + 3 at 2000 x 2000 and 1000 x 500,
    the small fit, the learned proposer, the comparison data and successive
    components."""
    import numpy as np
    import torch

    from paper_2402_16712_gb300 import autotune, datagen, l1line
    out = {}
    # lambda path: n=1000, m=500 float32, 32 lambdas in one fit
    X, lams, _ = datagen.lambda_path("float32")
    n, m = X.shape
    Xd = torch.from_numpy(X).to(dev)
    ws = l1line.Workspace.for_shape(torch.float32, n, m, lams.size, dev)
    res = (torch.empty((lams.size, m), dtype=torch.float32, device=dev),
           torch.empty(lams.size, dtype=torch.float64, device=dev),
           torch.empty(lams.size, dtype=torch.int32, device=dev))
    with torch.cuda.stream(stream):
        l1line.fit(Xd, lams, workspace=ws, stream=stream, out=res)
        tuning = autotune.apply(torch.float32, n, m, lams.size, flush=flush,
                                run=lambda: l1line.fit(Xd, lams, workspace=ws, stream=stream,
                                                       out=res))
        l1line.fit(Xd, lams, workspace=ws, stream=stream, out=res)
    stream.synchronize()
    launches = l1line.last_launch_count()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        l1line.fit(Xd, lams, workspace=ws, stream=stream, out=res)
    ms = _replay_ms(g, stream, 10, flush)
    l1line.set_tuning(None)
    if l1line.status(ws, stream) != l1line.OK:
        raise SystemExit("lambda-path fit failed on the device")
    pl = m * (m - 1) * lams.size
    out["lambda_path"] = {
        "workload": f"n={n}, m={m} float32, {lams.size} lambdas logspace(-3,1), one fit "
                    "(one pair launch for all lambdas), CUDA graph replay, L2 flushed",
        "ms_per_step": ms, "pair_lambdas_per_s": pl / (ms * 1e-3),
        "fits_per_s": lams.size / (ms * 1e-3), "gpu_launches_per_step": launches,
        "tuning": tuning}
    del Xd, ws, res, g
    # Algorithm 2 over every (jhat, k) pair and Algorithm 3 on top of it:
    # the 2000 x 2000 matrix (its lambda = 0 scan under the headline shape's
    # cached tuning) and the 1000 x 500 lambda-path matrix
    X, _, _ = datagen.paper_size("float32")
    ptune = autotune.apply(torch.float32, 2000, 2000, 1)
    big = measure_paths(dev, stream, flush, X)
    l1line.set_tuning(None)
    out["lambda_paths"] = {
        "workload": "Algorithm 2 for every (jhat, k) pair of the 2000 x 2000 float32 matrix: "
                    "exact lambda = 0 scan, count pass, offsets scan, write pass (L2 flushed, "
                    "CUDA events, output buffers allocated beforehand)",
        "ms_per_step": big["alg2_ms"], "breakpoints": big["entries"],
        "breakpoints_per_s": big["entries"] / (big["alg2_ms"] * 1e-3),
        "pairs_per_s": 2000 * 1999 / (big["alg2_ms"] * 1e-3), "tuning": ptune,
        "roofline": path_roofline(2000, 2000, big["entries"], big["alg2_ms"], 4)}
    out["solution_path_2000"] = {
        "workload": "Algorithms 2 and 3 on the 2000 x 2000 float32 matrix: every pair's path "
                    "with residuals, per-jhat objectives, lower envelope (CUDA events, output "
                    "buffers allocated beforehand, L2 flushed)",
        "ms_per_step": big["alg2_res_ms"] + big["alg3_ms"], "alg2_with_residuals_ms":
        big["alg2_res_ms"], "alg3_ms": big["alg3_ms"], "pieces": big["pieces"],
        "breakpoints": big["entries"]}
    X, _, _ = datagen.lambda_path("float32")
    small = measure_paths(dev, stream, flush, X)
    out["solution_path"] = {
        "workload": "Algorithms 2 and 3 on the n=1000, m=500 float32 lambda-path matrix: every "
                    "pair's path with residuals, per-jhat objectives, lower envelope (CUDA "
                    "events, output buffers allocated beforehand, L2 flushed)",
        "ms_per_step": small["alg2_res_ms"] + small["alg3_ms"],
        "alg2_with_residuals_ms": small["alg2_res_ms"], "alg3_ms": small["alg3_ms"],
        "pieces": small["pieces"], "jhat_star": small["jhat_star"]}
    # uneven batch: 256 instances, n~U[100,5000], m~U[10,500], lambda=0.2
    batch = datagen.uneven_batch(256)
    Xs = [torch.from_numpy(Xb).to(dev) for Xb, _ in batch]
    bat = l1line.Batched(Xs, [lb for _, lb in batch], device=dev)
    with torch.cuda.stream(stream):
        bat.run(stream)
        nmax = max(int(Xb.shape[0]) for Xb, _ in batch)
        mmax = max(int(Xb.shape[1]) for Xb, _ in batch)
        btune = autotune.apply(torch.float32, nmax, mmax, len(batch), kind="batch",
                               run=lambda: bat.run(stream))
        bat.run(stream)
    stream.synchronize()
    launches = l1line.last_launch_count()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        bat.run(stream)
    ms = _replay_ms(g, stream, 5)
    l1line.set_tuning(None)
    if bat.status(stream) != l1line.OK:
        raise SystemExit("batched fit failed on the device")
    pairs = int(sum(int(Xb.shape[1]) * (int(Xb.shape[1]) - 1) for Xb, _ in batch))
    out["uneven_batch"] = {
        "workload": "256 float32 instances, n~U[100,5000], m~U[10,500], lambda=0.2, one "
                    "persistent pair launch per size class, CUDA graph replay (inputs 658 MB "
                    "> L2)",
        "ms_per_step": ms, "fits_per_s": len(batch) / (ms * 1e-3),
        "pairs_per_s": pairs / (ms * 1e-3), "gpu_launches_per_step": launches,
        "tuning": btune}
    del Xs, bat, g
    out["small_fit"] = measure_small_fit(dev, stream)
    out["learned_topk"] = measure_learned(dev, stream, flush)
    for key, fn in (("comparison_suite", measure_comparison), ("components", measure_components),
                    ("tall_fit", measure_tall)):
        try:
            out[key] = fn(dev, stream, flush)
        except Exception as e:  # context lines only: never cost the headline
            out[key] = {"error": f"{type(e).__name__}: {e}"}
    return out


def path_roofline(n, m, entries, ms, es):
    """Algorithm 2's count and write passes against two ceilings: HBM (the
    bytes the write pass stores: lambda (8) and value (es) per breakpoint, a
    length (4) and an offset (8) per pair, against the measured copy
    bandwidth) and issue (two passes over the n rows of every pair at 6
    lane-instructions per row: load, multiply by the staged reciprocal, key,
    two compares, count or list; against 152 SMs x 128 lanes x 2070 MHz)."""
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    pairs = m * (m - 1)
    wbytes = entries * (8 + es) + m * m * (4 + 8)
    instr = 2 * 6 * n * pairs
    alu_peak = SMS * LANES_PER_SM_CLK * SM_MAX_MHZ * 1e6
    t = ms * 1e-3
    ce = {"hbm": {"achieved": wbytes / t / 1e9, "peak": hbm, "unit": "GB/s",
                  "frac": wbytes / t / 1e9 / hbm, "traffic_bytes": wbytes,
                  "peak_source": "MEASURED_PEAKS.json" if peaks else "fallback 6.8 TB/s"},
          "alu": {"achieved": instr / t / 1e12, "peak": alu_peak / 1e12, "unit": "Tinstr/s",
                  "frac": instr / t / alu_peak, "instructions": instr}}
    bound = max(ce, key=lambda c: wbytes / (hbm * 1e9) if c == "hbm" else instr / alu_peak)
    return {"bound": bound, **{k: ce[bound][k] for k in ("achieved", "peak", "unit", "frac")},
            "ceilings": ce}


def measure_paths(dev, stream, flush, X, reps=3):
    """Algorithm 2 (count + write, with and without residuals) and Algorithm 3
    (the envelope) of X through the library's entry points, each timed with
    CUDA events on the launching stream, L2 flushed before each; the output
    buffers are sized by one untimed run first, so no allocation or host read
    of a size lies inside a timed region."""
    import ctypes

    import torch

    from paper_2402_16712_gb300 import l1line
    lib = l1line.load()
    Xd = torch.from_numpy(X).to(dev)
    n, m = X.shape
    pws = l1line.path_workspace(Xd.dtype, n, m, dev)
    with torch.cuda.stream(stream):
        st, jh, I, S, V = l1line.solution_path(Xd, stream=stream)
        off, lam, v, ln, _, res = l1line.paths(Xd, workspace=pws, stream=stream, residuals=True)
    stream.synchronize()
    entries = int(off[m * m].item())
    pieces = int(st.numel())
    cap = pieces
    nb = int(lib.l1line_solution_path_workspace_bytes(m, entries))
    sws = l1line.Workspace(nb, dev)
    o_st = torch.empty(cap, dtype=torch.float64, device=dev)
    o_jh = torch.empty(cap, dtype=torch.int32, device=dev)
    o_I = torch.empty(cap, dtype=torch.float64, device=dev)
    o_S = torch.empty(cap, dtype=torch.float64, device=dev)
    o_v = torch.empty((cap, m), dtype=Xd.dtype, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    P = ctypes.c_void_p
    sp = P(stream.cuda_stream)
    f32 = Xd.dtype == torch.float32
    count = lib.l1line_path_count_f32 if f32 else lib.l1line_path_count_f64
    write = lib.l1line_path_write_f32 if f32 else lib.l1line_path_write_f64
    solve = lib.l1line_solution_path_f32 if f32 else lib.l1line_solution_path_f64

    def ok(rc, what):
        if rc != l1line.OK:
            raise SystemExit(f"{what}: {l1line.status_string(rc)}")

    def alg2(with_res):
        ok(count(Xd.data_ptr(), n, m, off.data_ptr(), P(pws.ptr), pws.nbytes, sp), "path count")
        ok(write(Xd.data_ptr(), n, m, off.data_ptr(), lam.data_ptr(), v.data_ptr(),
                 P(res.data_ptr()) if with_res else None, ln.data_ptr(), P(pws.ptr), pws.nbytes,
                 sp), "path write")

    def alg3():
        ok(solve(m, off.data_ptr(), lam.data_ptr(), v.data_ptr(), res.data_ptr(), ln.data_ptr(),
                 entries, o_st.data_ptr(), o_jh.data_ptr(), o_I.data_ptr(), o_S.data_ptr(),
                 o_v.data_ptr(), cnt.data_ptr(), cap, P(sws.ptr), sws.nbytes, sp),
           "solution path")

    def timed(fn):
        t = []
        for _ in range(reps):
            flush.fill_(6)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                a.record(stream)
                fn()
                b.record(stream)
            stream.synchronize()
            t.append(a.elapsed_time(b))
        return statistics.median(t)

    alg2(True)
    alg3()
    r = {"alg2_ms": timed(lambda: alg2(False)), "alg2_res_ms": timed(lambda: alg2(True)),
         "alg3_ms": timed(alg3), "entries": entries, "pieces": pieces,
         "jhat_star": sorted({int(x) for x in jh.tolist()})}
    if l1line.status(pws, stream) != l1line.OK or l1line.status(sws, stream) != l1line.OK:
        raise SystemExit("path enumeration failed on the device")
    if int(cnt.item()) != pieces:
        raise SystemExit("solution path piece count changed between runs")
    return r


def measure_components(dev, stream, flush, ncomp=3, steps=5):
    """Successive components: ncomp fits of the 1000 x 500 float32 lambda-path
    matrix at lambda = 0.5, each on the previous residual x_i - x_ijhat v (one
    library call; CUDA events around each call, L2 flushed before it)."""
    import torch

    from paper_2402_16712_gb300 import datagen, l1line

    l1line.set_tuning(None)  # the planner's launch
    X, _, _ = datagen.lambda_path("float32")
    Xd = torch.from_numpy(X).to(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    with torch.cuda.stream(stream):
        _, _, _, ws = l1line.components(Xd, 0.5, ncomp, stream=stream)
        for _ in range(2):
            l1line.components(Xd, 0.5, ncomp, workspace=ws, stream=stream)
        for a, b in ev:
            flush.fill_(3)
            a.record(stream)
            _, _, js, _ = l1line.components(Xd, 0.5, ncomp, workspace=ws, stream=stream)
            b.record(stream)
    stream.synchronize()
    if l1line.status(ws, stream) != l1line.OK:
        raise RuntimeError("components failed on the device")
    ms = statistics.median(a.elapsed_time(b) for a, b in ev)
    n, m = X.shape
    return {"workload": f"{ncomp} successive components of the n={n}, m={m} float32 "
                        "lambda-path matrix at lambda=0.5 (fit, deflate, repeat), one library "
                        "call, L2 flushed",
            "ms_per_step": ms, "components_per_s": ncomp / (ms * 1e-3),
            "pairs_per_s": ncomp * m * (m - 1) / (ms * 1e-3),
            "jhat_star": [int(j) for j in js.tolist()],
            "gpu_launches_per_step": l1line.last_launch_count()}


def measure_tall(dev, stream, flush, n=1_000_000, m=16, steps=5):
    """One fit of a tall matrix: n = 10^6 rows, m = 16, float32, the planted
    model (3-sparse v*, Laplace(0, 0.1), 5% N(0, 100 I) outlier rows) drawn on
    the device, lambda = 0.5.  n is beyond the shared-memory pair kernel, so
    the global-memory cluster path runs.  CUDA events around the whole fit and,
    through the library's hook, around the pair-stage launch; L2 flushed before
    each step.  Ceiling: every pass of that launch reads both columns (float
    keys: 3 descent passes and the residual pass), against the L2 read probe."""
    import torch

    from paper_2402_16712_gb300 import datagen, l1line

    X, _, _ = datagen.planted_torch(datagen.Planted(n, m, 3, 0.1, 0.05, 10.0, 7, "float32"), dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    with torch.cuda.stream(stream):
        for e in kev:  # the library records these on its stream: make them valid first
            e[0].record(stream)
            e[1].record(stream)
        _, _, _, ws = l1line.fit(X, [0.5], stream=stream)
        l1line.fit(X, [0.5], workspace=ws, stream=stream)
        for (a, b), (ka, kb) in zip(ev, kev):
            flush.fill_(5)
            l1line.profile_events(ka, kb)
            a.record(stream)
            _, obj, js, _ = l1line.fit(X, [0.5], workspace=ws, stream=stream)
            b.record(stream)
            l1line.profile_events(None, None)
    stream.synchronize()
    if l1line.status(ws, stream) != l1line.OK:
        raise RuntimeError("tall fit failed on the device")
    launches = l1line.last_launch_count()
    ms = statistics.median(a.elapsed_time(b) for a, b in ev)
    kms = statistics.median(a.elapsed_time(b) for a, b in kev)
    pairs = m * (m - 1)
    ldn = (n + 127) // 128 * 128
    streamed = pairs * 4 * 2 * 4 * ldn
    l2_gbs, _ = measure_ceilings(dev, stream)
    return {"workload": f"one fit of n={n}, m={m} float32 (planted model drawn on the device, "
                        "lambda=0.5): rows beyond the shared-memory pair kernel, global-memory "
                        "cluster path; CUDA events, L2 flushed",
            "ms_per_step": ms, "pairs_per_s": pairs / (ms * 1e-3),
            "pair_rows_per_s": pairs * n / (ms * 1e-3), "pair_stage_ms": kms,
            "jhat_star": int(js.item()), "objective": float(obj.item()),
            "roofline": {"bound": "l2", "achieved": streamed / (kms * 1e-3) / 1e9,
                         "peak": l2_gbs, "unit": "GB/s",
                         "frac": streamed / (kms * 1e-3) / 1e9 / l2_gbs,
                         "basis": "4 passes x 2 columns x 4 bytes x ldn per pair, against the "
                                  "L2 read probe of this run"},
            "gpu_launches_per_step": launches}


def measure_comparison(dev, stream, flush, steps=5):
    """The comparison experiment's data (30 float64 datasets of 100 x 100,
    five seeds per outlier count 1..6) with a sparsity sweep of 8 lambdas
    each, all in one batched call; CUDA events around each call, L2 flushed
    before it."""
    import numpy as np
    import torch

    from paper_2402_16712_gb300 import datagen, l1line

    l1line.set_tuning(None)  # the planner's launch
    Xs = datagen.comparison_suite("float64")
    lam = np.array([0.0, 5.0, 20.0, 50.0, 100.0, 200.0, 400.0, 800.0])
    bat = l1line.Batched([torch.from_numpy(X).to(dev) for X in Xs], [lam.copy() for _ in Xs],
                         device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    with torch.cuda.stream(stream):
        for _ in range(3):
            bat.run(stream)
        for a, b in ev:
            flush.fill_(2)
            a.record(stream)
            bat.run(stream)
            b.record(stream)
    stream.synchronize()
    if bat.status(stream) != l1line.OK:
        raise RuntimeError("batched fit failed on the device")
    ms = statistics.median(a.elapsed_time(b) for a, b in ev)
    fits = len(Xs) * lam.size
    pairs = sum(X.shape[1] * (X.shape[1] - 1) for X in Xs) * lam.size
    return {"workload": "the comparison experiment's data: 30 float64 datasets of 100 x 100 "
                        "(five seeds per outlier count 1..6), 8 lambdas each, one batched "
                        "call, L2 flushed",
            "ms_per_step": ms, "fits_per_s": fits / (ms * 1e-3),
            "pair_lambdas_per_s": pairs / (ms * 1e-3),
            "gpu_launches_per_step": l1line.last_launch_count()}


def measure_small_fit(dev, stream, replays=200):
    """The smallest workload: n=200, m=20 float64, lambda=0.1; one fit captured
    in a CUDA graph and replayed back to back (latency-bound; the 32 KB input
    stays in L2, no flush)."""
    import torch

    from paper_2402_16712_gb300 import datagen, l1line
    X, lams, _ = datagen.one_fit_small("float64")
    n, m = X.shape
    Xd = torch.from_numpy(X).to(dev)
    ws = l1line.Workspace.for_shape(torch.float64, n, m, 1, dev)
    res = (torch.empty((1, m), dtype=torch.float64, device=dev),
           torch.empty(1, dtype=torch.float64, device=dev),
           torch.empty(1, dtype=torch.int32, device=dev))
    with torch.cuda.stream(stream):
        for _ in range(3):
            l1line.fit(Xd, lams, workspace=ws, stream=stream, out=res)
    stream.synchronize()
    launches = l1line.last_launch_count()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        l1line.fit(Xd, lams, workspace=ws, stream=stream, out=res)
    ms = _replay_ms(g, stream, replays)
    if l1line.status(ws, stream) != l1line.OK:
        raise SystemExit("small fit failed on the device")
    return {"workload": f"n={n}, m={m} float64, 4-sparse v*, Laplace(0,0.05), 10% N(0,25 I) "
                        "outliers, lambda=0.1; CUDA graph replayed back to back",
            "us_per_fit": ms * 1e3, "fits_per_s": 1.0 / (ms * 1e-3),
            "pairs_per_s": m * (m - 1) / (ms * 1e-3), "gpu_launches_per_step": launches}


def measure_learned(dev, stream, flush, count=32, Ks=(32, 128)):
    """The learned top-K path against the full scan on a sample of held-out
    5000 x 1000 float32 instances (the committed network; the 200-instance
    evaluation is the proposer module's `eval`).  Times are CUDA events with L2
    flushed; zero regret = the learned path's objective equals the scan's bit
    for bit."""
    import numpy as np
    import torch

    from paper_2402_16712_gb300 import datagen, l1line, proposer
    mlp = proposer.network(dev)
    n, m = 5000, 1000
    ws = l1line.proposed_workspace(torch.float32, n, m, 1, dev)

    def timed(fn):
        flush.fill_(5)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            r = fn()
            e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1), r

    full_ms, learned_ms, hits = [], {K: [] for K in Ks}, {K: 0 for K in Ks}
    for q in range(count):
        X, lams, _ = datagen.proposer_instance(datagen.PROPOSER_HELDOUT_SEED0 + q, n=n, m=m)
        Xd = torch.from_numpy(X).to(dev)
        with torch.cuda.stream(stream):
            l1line.fit(Xd, lams, workspace=ws, stream=stream)
        ms, (v, obj, js, _) = timed(lambda: l1line.fit(Xd, lams, workspace=ws, stream=stream))
        full_ms.append(ms)
        z_full = obj.cpu().numpy().copy()
        for K in Ks:
            with torch.cuda.stream(stream):
                l1line.fit_proposed(Xd, lams, mlp, K, workspace=ws, stream=stream)
            ms, (v2, obj2, js2, _, _) = timed(
                lambda: l1line.fit_proposed(Xd, lams, mlp, K, workspace=ws, stream=stream))
            learned_ms[K].append(ms)
            hits[K] += int(np.array_equal(obj2.cpu().numpy().view(np.int64),
                                          z_full.view(np.int64)))
    if l1line.status(ws, stream) != l1line.OK:
        raise SystemExit("learned path failed on the device")
    fm = float(np.median(full_ms))
    return {"workload": f"{count} held-out planted instances n={n}, m={m} float32, lambda=0.2 "
                        "(seeds from the held-out range); learned path = features, network, "
                        "top-K, exact fit of the K candidates",
            "full_scan_ms": fm,
            "K": {str(K): {"ms": float(np.median(learned_ms[K])),
                           "speedup_vs_full_scan": fm / float(np.median(learned_ms[K])),
                           "zero_regret_fraction": hits[K] / count} for K in Ks}}


def run_sharded(args):
    """--sharded: the headline is one 2000 x 2000 fit split over this job's
    ranks by jhat (strong scaling); see measure_sharded."""
    import torch

    from paper_2402_16712_gb300 import l1line
    rank, world, local = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if rank == 0 or world == 1:
        import __graft_entry__
        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
    l1line.load()
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    clk = Clocks(dev.index)
    clk.start()
    r = measure_sharded(dev, stream, dist, args.steps, args.warmup, flush)
    clocks = clk.stop()
    launches = l1line.last_launch_count()
    if rank == 0:
        line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "n": N_ROWS, "m": N_COLS, "lambda": LAMBDA,
                           "pairs_per_fit": N_COLS * (N_COLS - 1),
                           "parallelism": f"jhat-sharded x{world} (one fit over all ranks)",
                           "l2": "flushed before every timed step (512 MiB write)"},
                "fits_per_s": r["fits_per_s"], "identical_to_one_gpu": r["identical_to_one_gpu"],
                "gpu_launches": launches * args.steps, "clocks": clocks}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_profile_case(args):
    """A plain run of a few fits at a given shape (no timing), for ncu."""
    import torch

    from paper_2402_16712_gb300 import datagen, l1line
    import __graft_entry__
    __graft_entry__.build()
    dt = "float32" if args.dtype == "f32" else "float64"
    X, lams, _ = datagen.paper_size(dt, n=args.n, m=args.m)
    Xd = torch.from_numpy(X).cuda()
    ws = l1line.Workspace.for_shape(Xd.dtype, args.n, args.m, 1)
    if args.d0:
        l1line.set_tuning({"d0": args.d0})
    for _ in range(args.fits):
        l1line.fit(Xd, lams, workspace=ws)
    rc = l1line.status(ws)
    plan = (l1line.plan(Xd.dtype, args.n, args.m) if args.n <= l1line.max_rows(Xd.dtype)
            else "global-memory cluster path")
    print(f"profile case n={args.n} m={args.m} {dt} d0={args.d0 or 'planner'}: "
          f"plan={plan} status={l1line.status_string(rc)}")
    return 0 if rc == l1line.OK else 1


def run_profile_batch(args):
    """A plain run of the 256-instance uneven batch (no timing, no graph), for
    a launch list: one persistent pair launch per size class."""
    import torch

    from paper_2402_16712_gb300 import datagen, l1line
    import __graft_entry__
    __graft_entry__.build()
    batch = datagen.uneven_batch(256)
    Xs = [torch.from_numpy(Xb).cuda() for Xb, _ in batch]
    bat = l1line.Batched(Xs, [lb for _, lb in batch])
    for _ in range(args.fits):
        bat.run()
    rc = bat.status()
    print(f"profile batch: 256 instances, launches per call {l1line.last_launch_count()}, "
          f"status={l1line.status_string(rc)}")
    return 0 if rc == l1line.OK else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the headline line (skip the lambda-path, path, batch, small-fit, "
                         "proposer, comparison and components lines)")
    ap.add_argument("--sharded", action="store_true",
                    help="headline = one 2000 x 2000 fit split over the ranks by jhat (strong "
                         "scaling, NCCL argmin), checked bit for bit against the one-GPU fit")
    ap.add_argument("--profile-batch", action="store_true",
                    help="run --fits plain calls of the 256-instance uneven batch (for ncu)")
    ap.add_argument("--profile-case", action="store_true",
                    help="run --fits plain fits of an n x m instance (for ncu), no timing")
    ap.add_argument("--n", type=int, default=N_ROWS)
    ap.add_argument("--m", type=int, default=N_COLS)
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--fits", type=int, default=2)
    ap.add_argument("--d0", type=int, default=0,
                    help="--profile-case: first-bracket half-width (0 = the planner's)")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args)
    if args.profile_batch:
        return run_profile_batch(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.sharded:
        return run_sharded(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
