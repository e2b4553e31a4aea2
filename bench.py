#!/usr/bin/env python
"""Benchmark of the eigenvector-eigenvalue identity path on GB300.

Default workload: one FP64 matrix n = 1024 with a planted spectrum (Q from a
Householder QR of a seeded Gaussian matrix, eigenvalues uniform on [-1, 1] with
minimum gap 1e-4), the full 1024 x 1024 grid |v_ij|^2.  One step = one call of
eeid_components over that grid (all five phases: Householder reduction of A and
its 1024 minors, bisection of A, denominators, bisection of the minors, Eq. 1).
Metric: |v_ij|^2 components per second (higher is better).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

For N > 1 launch under torchrun: each rank runs its own replica of the workload
(weak scaling, no data-path collective); rank 0 prints one JSON line with the
aggregate over ranks and the max time over ranks.  --impl reference times the CPU
oracle (long double, host cores) on a bounded sample of the same workload.
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

METRIC = "|v_ij|^2 components/s at <=1e-10 err"
UNIT = "components/s"
WORKLOAD = ("planted1024: one FP64 n=1024 planted-spectrum matrix (lam uniform on [-1,1], "
            "min gap 1e-4), full 1024x1024 |v_ij|^2 grid")
N = 1024

# FP64 peak of one GB300 derived from its unit counts and clock: 152 SMs x 2 FP64
# FMA lanes/clk/SM (4 flop/clk/SM; 1.25 TFLOP/s nominal) x 2.07 GHz max SM clock.
FP64_PEAK_GFLOPS = 152 * 4 * 2.07
# Algorithmic work of the dominant kernel (Householder tridiagonalisation, 4/3 m^3
# flops per m x m matrix) for one step: A (m = n) plus n minors (m = n - 1).
TRIDIAG_FLOPS = 4.0 / 3.0 * (N ** 3 + N * (N - 1) ** 3)

# DRAM traffic of the tridiagonalisation phase of one step (all its launches), from an
# ncu capture scaled by the work (profiles/), valid only while the kernel's device code
# is unchanged: sha256 of csrc/tridiag.cu up to the end of its anonymous namespace,
# which holds every device function (host-side launch code below it may change),
# followed by the header of the tile split it includes.
TRIDIAG_TRAFFIC = {"bytes_per_launch": 3.194e12,
                   "device_code_sha256": "84f7fdfb39d7840490ff8bf6b16caa3edd12bbbc21c6df6b3b845c864c2feb23"}


def device_code_sha(path: str, *headers: str) -> str:
    """sha256 of a kernel source up to the end of its anonymous namespace (the device code)
    and of the headers given."""
    with open(path) as f:
        text = f.read()
    text = text[: text.index("}  // namespace\n")]
    for h in headers:
        with open(h) as f:
            text += f.read()
    return hashlib.sha256(text.encode()).hexdigest()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_dist(world: int, backend: str):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend)
    return dist if world > 1 else None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x: float, device=None) -> float:
    """Max of a float over all ranks (timing aggregation, not a data-path collective)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(units_per_rank_per_step: float, world: int, steps: int, max_ms: float) -> float:
    """Whole-job throughput: units all ranks processed / max time over ranks."""
    return units_per_rank_per_step * world * steps / (max_ms / 1e3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle leg

def oracle_sample(planted, target_s: float = 15.0):
    """Time the CPU oracle on a bounded sample of the workload: the components of
    whole columns j, i.e. the minor eigenvalues of M_j (roots of the secular equation
    from the known (lam, Q), long double) followed by Eq. 1 in long double for all i.
    Returns (components/s, columns, seconds, cores)."""
    import numpy as np

    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    lam, Q = planted.lam, planted.Q
    # one column first to size the sample, then as many as fit in the target
    t0 = time.perf_counter()
    mu = oracle.secular_minor_eigvals(lam, Q, [0])
    oracle.identity(lam, mu)
    one = time.perf_counter() - t0
    ncols = int(max(1, min(N - 1, (target_s / max(one, 1e-3)) * cores)))
    ncols = max(cores, (ncols // cores) * cores) if ncols >= cores else ncols
    cols = np.arange(1, 1 + min(ncols, N - 1))
    t0 = time.perf_counter()
    mu = oracle.secular_minor_eigvals(lam, Q, cols)
    oracle.identity(lam, mu)
    dt = time.perf_counter() - t0
    return N * cols.size / dt, int(cols.size), dt, cores


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    from paper_2002_04989_gb300 import inputs
    p = inputs.planted1024()
    vals, secs, cols = [], [], 0
    for step in range(args.warmup + args.steps):
        v, c, dt, cores = oracle_sample(p, target_s=min(10.0, 100.0 / max(1, args.steps)))
        if step >= args.warmup:
            vals.append(v)
            secs.append(dt)
            cols = c
    value = statistics.mean(vals)
    sample = (f"{cols} columns j of the n=1024 planted matrix per step: minor eigenvalues by "
              f"secular-equation bisection from the planted (lam, Q), then Eq. 1, long double, "
              f"OpenMP over columns")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n": N},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU leg

def run_gpu(args, world, rank, local):
    import numpy as np
    import torch

    from paper_2002_04989_gb300 import eeid, inputs

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    dev = torch.device("cuda", local)
    p = inputs.planted1024()
    A = torch.from_numpy(p.A).to(dev)
    out = torch.empty((N, N), dtype=torch.float64, device=dev)
    lam = torch.empty(N, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    ctx = eeid.Context(local)
    stream = torch.cuda.current_stream(dev)

    def step():
        ctx.eeid_components(A, out=out, lam=lam, stream=stream)
        flush.fill_(step.counter & 0xff)   # evict L2 between steps
        step.counter += 1
    step.counter = 0

    for _ in range(args.warmup):
        step()
    st = ctx.eeid_sync(stream)
    # accuracy of the timed configuration against the planted closed form
    err = float(np.max(np.abs(out.cpu().numpy() - (p.Q * p.Q).T)))

    ctx.eeid_set_timing(True)
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    barrier(dist)
    torch.cuda.synchronize()
    clocks.start()
    l0 = ctx.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    tri_ms, phases = [], []
    e0.record(stream)
    for _ in range(args.steps):
        step()                            # no host wait between steps
    e1.record(stream)
    torch.cuda.synchronize()
    # the per-phase events of the last timed step (recorded inside the timed region)
    ph = ctx.eeid_phase_times()
    phases.append(ph)
    tri_ms.append(ph["tridiag"])
    barrier(dist)
    torch.cuda.synchronize()
    launches = ctx.launch_count() - l0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    max_ms = max_over_ranks(dist, ms, dev)
    value = aggregate_value(N * N, world, args.steps, max_ms)
    ctx.eeid_set_timing(False)

    # ---- end to end: host buffers through the public C ABI (copies in the region)
    hA = torch.from_numpy(p.A).pin_memory().numpy()
    hout = torch.empty((N, N), dtype=torch.float64).pin_memory().numpy()
    hlam = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
    ctx.eeid_components_host(hA, out=hout, lam=hlam)
    barrier(dist)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.eeid_components_host(hA, out=hout, lam=hlam)
        flush.fill_(1)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier(dist)
    e2e_max = max_over_ranks(dist, e2e_s * 1e3, dev)
    e2e_value = aggregate_value(N * N, world, args.steps, e2e_max)

    # ---- roofline of the dominant kernel (tridiagonalisation), FP64 ALU bound
    tri_avg = statistics.mean(tri_ms)
    achieved = TRIDIAG_FLOPS / (tri_avg / 1e3) / 1e12
    peak = FP64_PEAK_GFLOPS / 1e3
    csrc = os.path.join(ROOT, "paper_2002_04989_gb300", "csrc")
    sha = device_code_sha(os.path.join(csrc, "tridiag.cu"), os.path.join(csrc, "tile_split.h"))
    traffic = (TRIDIAG_TRAFFIC["bytes_per_launch"]
               if TRIDIAG_TRAFFIC["device_code_sha256"] == sha else None)
    phase_avg = {k: round(statistics.mean(ph[k] for ph in phases), 3) for k in phases[0]}

    if rank != 0:
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, c, dt, cores = oracle_sample(p)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": (f"{c} columns j of the same matrix ({c * N} components, {dt:.1f} s): "
                          f"minor eigenvalues by secular-equation bisection from the planted "
                          f"(lam, Q), then Eq. 1, long double, OpenMP over columns")}
    workloads = None
    if world == 1 and not args.no_workloads:
        # the other workloads, each timed after the headline's timed region, with its own
        # events, clocks and roofline (goe64: 3+10 calls; batch4096: 3+2 batched steps and
        # one plain pass; planted4096 and vectors1024: 1+1 steps; serving: one rate)
        workloads = {}
        ctx.eeid_tune_reset()
        for name, st_, wu in (("goe64", 10, 3), ("batch4096", 2, 3), ("planted4096", 1, 1),
                              ("vectors1024", 1, 1), ("herm1024", 1, 1), ("single4002", 3, 1)):
            try:
                workloads[name] = workload_record(name, ctx, dev, stream, st_, wu, local)
            except Exception as ex:   # a failed sub-record must not hide the headline
                workloads[name] = {"error": repr(ex)}
            ctx.eeid_tune_reset()
        try:
            workloads["serving"] = serving_record(local, args.serving_requests, [2.0])
        except Exception as ex:
            workloads["serving"] = {"error": repr(ex)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded planted spectrum; no dataset)",
        "config": {"workload": WORKLOAD, "n": N, "components_per_step_per_gpu": N * N,
                   "l2": "flushed between steps (256 MiB write, inside the timed region)",
                   "parallelism": f"replicas x{world} (weak scaling, no collective)"},
        "roofline": {"bound": "alu",
                     "kernel": "k_tridiag (FP64 Householder, A + 1024 minors: 8-warp pair "
                               "rounds + 16-warp tail; time = the phase's span in the last "
                               "timed step, CUDA events)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": "derived: 152 SM x 4 FP64 flop/clk x 2.07 GHz "
                                    "(recipe: 1.25 TFLOP/s nominal)"},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * N * N,
                "d2h_bytes_per_step": 8 * N * N + 8 * N},
        "clocks": clk,
        "gpu_launches": launches,
        "phases_ms": phase_avg,
        "max_abs_err_vs_QoQ": err,
        "status": st,
        "workloads": workloads,
    }
    print(json.dumps(line), flush=True)
    return 0


def tridiag_flops(sizes_and_cols) -> float:
    """4/3 m^3 per tridiagonalisation: A (m = n) and each requested minor (m = n-1)."""
    return sum(4.0 / 3.0 * (n ** 3 + nc * (n - 1) ** 3) for n, nc in sizes_and_cols)


def alu_roofline(flops: float, ms: float, kernel: str) -> dict:
    achieved = flops / (ms / 1e3) / 1e12 if ms and ms > 0 else None
    peak = FP64_PEAK_GFLOPS / 1e3
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
            "traffic": None, "peak_source": "derived: 152 SM x 4 FP64 flop/clk x 2.07 GHz"}


def _timed(torch, stream, fn, steps):
    """CUDA-event time of `steps` calls of fn on `stream` (ms, whole span)."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def workload_record(name, ctx, dev, stream, steps, warmup, local=0):
    """One other workload, timed after the headline: goe64 (one small matrix, all
    minors), batch4096 (4096 matrices of uneven n in one batched call, against the plain
    one-call-per-matrix loop), planted4096 (n = 4096, 256 seeded columns) and vectors1024
    (signed eigenvectors of the planted n = 1024 matrix for 16 eigen-indices).  Returns a
    dict with its own CUDA-event timing, roofline, clocks and status."""
    import numpy as np
    import torch

    from paper_2002_04989_gb300 import inputs
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    rec = {}
    plain_step = None
    extra_steps = {}   # label -> another plan of the same step, timed once after the run
    phase_timed = True
    if name == "batch4096":
        # per-size kernel variants picked by the autotuner (cached per device model)
        tune_path = os.path.join(ROOT, "paper_2002_04989_gb300", "_build", "tune_table.txt")
        t0 = time.perf_counter()
        ctx.eeid_autotune(256, tune_path)
        rec["autotune_s"] = round(time.perf_counter() - t0, 2)
        rec["tune_table"] = open(tune_path).read().splitlines()[1:]
        mats = inputs.batch4096()
        sizes = [A.shape[0] for A in mats]
        big = torch.empty(sum(n * n for n in sizes), dtype=torch.float64, device=dev)
        outs = torch.empty(sum(n * n for n in sizes), dtype=torch.float64, device=dev)
        probs, off = [], 0
        big.copy_(torch.from_numpy(np.concatenate([A.reshape(-1) for A in mats])))
        for A in mats:
            n = A.shape[0]
            probs.append({"A": big[off:off + n * n].view(n, n),
                          "out": outs[off:off + n * n].view(n, n)})
            off += n * n
        units = float(sum(n * n for n in sizes))
        flops = tridiag_flops([(n, n) for n in sizes])

        def step():
            ctx.eeid_components_batched(probs, stream=stream)
            flush.fill_(1)

        def plain_step():
            for pr in probs:
                ctx.eeid_components(pr["A"], out=pr["out"], stream=stream)
            flush.fill_(1)
        workload = (f"batch4096: 4096 FP64 symmetric matrices, n log-uniform on [8,256] "
                    f"(sum n = {sum(sizes)}), thirds GOE / Wishart / Toeplitz(0,1), all components")
    elif name == "planted4096":
        pl, cols = inputs.planted4096()
        A = torch.from_numpy(pl.A).to(dev)
        out = torch.empty((4096, 256), dtype=torch.float64, device=dev)
        units = 4096.0 * 256
        flops = tridiag_flops([(4096, 256)])

        def step():
            ctx.eeid_components(A, cols=cols, out=out, stream=stream)
            flush.fill_(1)
        workload = ("planted4096: one FP64 n=4096 planted matrix (lam on [-10,10], min gap "
                    "1e-4), all i x 256 seeded columns j (256 minors of size 4095)")
    elif name == "vectors1024":
        pl = inputs.planted1024()
        A = torch.from_numpy(pl.A).to(dev)
        rows = np.unique(np.r_[0, 511, 1023,
                               np.random.default_rng(5).choice(1024, 13, replace=False)])
        out = torch.empty((rows.size, 1024), dtype=torch.float64, device=dev)
        units = float(rows.size * 1024)
        flops = None   # depends on the references chosen; filled in below

        def step():
            ctx.eeid_eigenvectors(A, rows=rows, out=out, stream=stream)
            flush.fill_(1)
        phase_timed = False
        workload = (f"vectors1024: signed eigenvectors (all 1024 components) of the planted "
                    f"n=1024 matrix for {rows.size} seeded eigen-indices")
    elif name == "single4002":
        pl = inputs.planted(4002, inputs.seed_for(inputs.CFG_PLANTED4096, 2), -1.0, 1.0, 1e-4)
        A = torch.from_numpy(pl.A).to(dev)
        out = torch.empty((1, 1), dtype=torch.float64, device=dev)
        units = 1.0
        flops = tridiag_flops([(4002, 1)])
        ij = (1234, 2001)

        def step():
            ctx.eeid_components(A, rows=[ij[0]], cols=[ij[1]], out=out, stream=stream)
            flush.fill_(1)

        def plain_step():
            ctx.eeid_set_clusters(0)
            step()
            ctx.eeid_set_clusters(2)

        def cluster_step():
            ctx.eeid_set_clusters(1)
            step()
            ctx.eeid_set_clusters(2)
        extra_steps["cluster_plan_16_ctas_per_matrix"] = cluster_step
        workload = ("single4002: one component |v_ij|^2 (i=1234, j=2001) of a planted FP64 "
                    "n=4002 matrix: A and one minor, group plan (latency mode: each reduction "
                    "on 76 CTAs); the paper's Table 1 task at n=4002 took 16.78 s on a 4-core "
                    "Xeon (context only)")
    elif name == "herm1024":
        pl = inputs.planted_herm(1024, inputs.seed_for(inputs.CFG_PLANTED1024, 7))
        A = torch.from_numpy(pl.A).to(dev)
        out = torch.empty((1024, 1024), dtype=torch.float64, device=dev)
        units = 1024.0 * 1024
        flops = 4.0 * tridiag_flops([(1024, 1024)])   # complex: 4 real FMA per complex FMA

        def step():
            ctx.eeid_components_herm(A, out=out, stream=stream)
            flush.fill_(1)
        workload = ("herm1024: one complex Hermitian n=1024 planted-spectrum matrix (unitary Q, "
                    "lam on [-1,1], min gap 1e-4), full 1024x1024 |v_ij|^2 grid")
    else:
        A = torch.from_numpy(inputs.goe64()).to(dev)
        out = torch.empty((64, 64), dtype=torch.float64, device=dev)
        units = 64.0 * 64
        flops = tridiag_flops([(64, 64)])

        def step():
            ctx.eeid_components(A, out=out, stream=stream)
            flush.fill_(1)
        workload = "goe64: one FP64 GOE matrix n=64 (seed 0), all minors, full 64x64 grid"

    for _ in range(warmup):
        step()
    st = ctx.eeid_sync(stream)
    if name == "planted4096":
        rec["max_abs_err_vs_QoQ"] = float(np.max(np.abs(out.cpu().numpy() - (pl.Q * pl.Q).T[:, cols])))
    if name == "single4002":
        rec["abs_err_vs_QoQ"] = float(abs(out.cpu().numpy()[0, 0] - pl.Q[ij[1], ij[0]] ** 2))
    if name == "herm1024":
        rec["max_abs_err_vs_absQ2"] = float(np.max(np.abs(out.cpu().numpy() - (np.abs(pl.Q) ** 2).T)))
    if name == "vectors1024":
        ref = pl.Q.T[rows]
        ref = ref * np.sign(ref[np.arange(rows.size), np.argmax(np.abs(ref), axis=1)])[:, None]
        rec["max_abs_err_vs_Q"] = float(np.max(np.abs(out.cpu().numpy() - ref)))
        R = ctx.eeid_vector_refs()
        rec["references"] = R
        flops = 4.0 / 3.0 * (1024 ** 3 + (1024 + R * 1023) * 1023 ** 3)
    ctx.eeid_set_timing(phase_timed)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = ctx.launch_count()
    phases = []

    ms = _timed(torch, stream, step, steps)
    if phase_timed:   # the last timed step's phase events
        phases.append(ctx.eeid_phase_times())
    clk = clocks.stop()
    launches = ctx.launch_count() - l0
    ctx.eeid_set_timing(False)
    phase_avg = ({k: round(statistics.mean(ph[k] for ph in phases), 3) for k in phases[0]}
                 if phases else None)
    if plain_step is not None:
        plain_step()
        pm = _timed(torch, stream, plain_step, 1)
        key = "one_cta_per_matrix" if name == "single4002" else "plain_one_call_per_matrix"
        rec[key] = {"value": units / (pm / 1e3), "ms_per_step": pm}
    for key, fn in extra_steps.items():
        fn()
        pm = _timed(torch, stream, fn, 1)
        rec[key] = {"value": units / (pm / 1e3), "ms_per_step": pm}
    if phase_avg:
        roof = alu_roofline(flops, phase_avg.get("tridiag", 0.0),
                            "k_tridiag (all tridiagonalisations of a step; time = the phase's span in the last timed step)")
    else:
        roof = alu_roofline(flops, ms / steps,
                            "all kernels of the call (reductions of A, its minors and the "
                            "rotated minors; time = the whole call)")
    base = {"workload": workload, "value": units * steps / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms / steps, "steps": steps, "warmup": warmup,
            "components_per_step": units, "roofline": roof, "clocks": clk,
            "gpu_launches": launches, "phases_ms": phase_avg, "status": st,
            "timing": "CUDA events on the launching stream; L2 flushed between steps"}
    base.update(rec)
    return base


def run_other(args, world, rank, local):
    """The line of one other workload (see workload_record)."""
    import torch

    from paper_2002_04989_gb300 import eeid
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    dev = torch.device("cuda", local)
    ctx = eeid.Context(local)
    stream = torch.cuda.current_stream(dev)
    barrier(dist)
    r = workload_record(args.workload, ctx, dev, stream, args.steps, args.warmup, local)
    max_ms = max_over_ranks(dist, r["ms_per_step"] * args.steps, dev)
    value = aggregate_value(r["components_per_step"], world, args.steps, max_ms)
    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": r.pop("workload"),
                       "components_per_step_per_gpu": r.pop("components_per_step"),
                       "l2": "flushed between steps (256 MiB write)"}}
    for k in ("value", "ms_per_step", "steps", "warmup"):
        r.pop(k)
    line.update(r)
    print(json.dumps(line), flush=True)
    return 0


def serving_record(local, nreq, rates, log=None):
    """Serving: a prefix of the seeded request stream (GOE or planted, n log-uniform
    on [16, 2048], all components or 1-64 random columns) arriving as a Poisson
    process, through the continuous-batching server and, for comparison, through the
    plain path (one request at a time in arrival order, host buffers, one context)."""
    import threading

    import numpy as np

    from paper_2002_04989_gb300 import eeid, inputs
    reqs = [inputs.serving_request(rid) for rid in range(nreq)]
    comps = [r.A.shape[0] * (r.A.shape[0] if r.cols is None else len(r.cols)) for r in reqs]
    work = sum(4.0 / 3.0 * (r.A.shape[0] ** 3 + (r.A.shape[0] if r.cols is None else len(r.cols))
                            * (r.A.shape[0] - 1) ** 3) for r in reqs)
    results = []

    def pct(xs, q):
        return float(np.percentile(np.asarray(xs), q))

    for rate in rates:
        arr = inputs.serving_arrivals(nreq, rate)
        clocks = ClockSampler(local)
        clocks.start()
        # ---- continuous batching
        lat, done_t = [None] * nreq, [0.0] * nreq
        with eeid.Server(local) as srv:
            tickets = [None] * nreq
            ready = threading.Semaphore(0)

            def collect():
                for k in range(nreq):
                    ready.acquire()
                    out, lam, st = srv.eeid_server_wait(tickets[k])
                    lat[k] = st["total_ms"]
                    done_t[k] = time.perf_counter()
            th = threading.Thread(target=collect)
            th.start()
            t0 = time.perf_counter()
            for k, r in enumerate(reqs):
                dt = t0 + arr[k] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                tickets[k] = srv.eeid_server_submit(r.A, cols=r.cols)
                ready.release()
            th.join()
            info = srv.eeid_server_info()
        span = max(done_t) - t0
        served = {"p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "value": sum(comps) / span,
                  "makespan_s": span, "fp64_tflops": work / span / 1e12,
                  "batches": info["batches_launched"],
                  "max_overlapping_batches": info["max_overlapping_batches"]}
        # ---- plain: one request at a time, arrival order
        ctx = eeid.Context(local)
        lat_p = []
        t0 = time.perf_counter()
        for k, r in enumerate(reqs):
            dt = t0 + arr[k] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            ctx.eeid_components_host(r.A, cols=r.cols)
            lat_p.append(1e3 * (time.perf_counter() - (t0 + arr[k])))
        span_p = time.perf_counter() - t0
        ctx.close()
        clk = clocks.stop()
        plain = {"p50_ms": pct(lat_p, 50), "p99_ms": pct(lat_p, 99), "value": sum(comps) / span_p,
                 "makespan_s": span_p, "fp64_tflops": work / span_p / 1e12}
        results.append({"rate_per_s": rate, "served": served, "plain": plain, "clocks": clk})
        if log is not None:
            print(json.dumps({"rate": rate, "served": served, "plain": plain}), file=log, flush=True)
    return {"workload": (f"serving: first {nreq} requests of the seeded stream (GOE or planted "
                         f"50:50, n log-uniform on [16,2048], all or 1-64 columns), Poisson "
                         f"arrivals"),
            "requests": nreq, "components": sum(comps), "tridiag_flops": work,
            "timing": "host wall clock from each arrival to its results in host memory",
            "sweep": results}


def run_serving(args, world, rank, local):
    import torch
    torch.cuda.set_device(local)
    rates = [float(r) for r in args.serving_rates.split(",")]
    rec = serving_record(local, args.serving_requests, rates, log=sys.stderr)
    if rank != 0:
        return 0
    best = max(rec["sweep"], key=lambda x: x["served"]["value"])
    line = {"metric": METRIC + "; serving p50/p99 latency vs plain GPU path",
            "value": best["served"]["value"], "unit": UNIT, "n_gpus": 1, "steps": len(rates),
            "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": rec["workload"], "requests": rec["requests"],
                       "components": rec["components"], "tridiag_flops": rec["tridiag_flops"]},
            "sweep": rec["sweep"]}
    print(json.dumps(line), flush=True)
    return 0


def run_profile_case(case: str) -> int:
    """Small, self-checking cases sized for an ncu capture (a few GB on the device):
    tridiag152 / tridiag304 = A plus the first 151 / 303 minors of the planted n=1024
    matrix (one / two CTAs per SM), called twice (its k_bisect, k_denominators and
    k_identity launches are the ones captured for those kernels); batch256 = the
    matrices of the uneven batch with n in (192, 256] (316 of them) in one batched call
    with the autotuned variants, graphs off, called twice; single2002 = one component of
    a planted n = 2002 matrix (the group plan: two groups of 76 CTAs), called twice;
    cluster2002 = the same on the cluster plan (two clusters of 16); herm512 = a complex
    Hermitian n = 512 matrix with 151 columns, called twice."""
    import numpy as np
    import torch

    from paper_2002_04989_gb300 import eeid, inputs
    ctx = eeid.Context(0)
    if case in ("single2002", "cluster2002"):
        # one component of a planted n = 2002 matrix: A and one minor, two groups of 76
        # CTAs (or two clusters of 16)
        ctx.eeid_set_clusters(2 if case == "single2002" else 1)
        pl = inputs.planted(2002, 2002, -1.0, 1.0, 1e-4)
        A = torch.from_numpy(pl.A).cuda()
        for _ in range(2):
            out = ctx.eeid_components(A, rows=[700], cols=[1500])
            ctx.eeid_sync()
        err = abs(float(out.cpu().numpy()[0, 0]) - pl.Q[1500, 700] ** 2)
        print(f"{case}: abs err vs Q o Q = {err:.3e}")
        return 0 if err <= 1e-10 else 1
    if case == "herm512":
        # complex Hermitian n = 512, 151 columns: 152 reductions, one CTA per SM
        pl = inputs.planted_herm(512, 512, -1.0, 1.0, 1e-4)
        A = torch.from_numpy(pl.A).cuda()
        cols = np.arange(151)
        for _ in range(2):
            out = ctx.eeid_components_herm(A, cols=cols)
            ctx.eeid_sync()
        err = float(np.max(np.abs(out.cpu().numpy() - (np.abs(pl.Q) ** 2).T[:, cols])))
        print(f"{case}: max abs err vs |Q|^2 = {err:.3e}")
        return 0 if err <= 1e-10 else 1
    if case == "batch256":
        tune_path = os.path.join(ROOT, "paper_2002_04989_gb300", "_build", "tune_table.txt")
        ctx.eeid_autotune(256, tune_path)
        ctx.eeid_set_graphs(False)
        mats = [A for A in inputs.batch4096() if 192 < A.shape[0] <= 256]
        probs = []
        for A in mats:
            n = A.shape[0]
            probs.append({"A": torch.from_numpy(A).cuda(),
                          "out": torch.empty((n, n), dtype=torch.float64, device="cuda")})
        for _ in range(2):
            ctx.eeid_components_batched(probs)
            ctx.eeid_sync()
        worst = max(float(np.max(np.abs(pr["out"].sum(dim=0).cpu().numpy() - 1.0))) for pr in probs)
        print(f"{case}: {len(mats)} matrices, worst column-sum deviation {worst:.3e}")
        return 0 if worst <= 1e-9 else 1
    p = inputs.planted1024()
    A = torch.from_numpy(p.A).cuda()
    cols = np.arange(151 if case == "tridiag152" else 303)
    for _ in range(2):
        out = ctx.eeid_components(A, cols=cols)
        ctx.eeid_sync()
    err = float(np.max(np.abs(out.cpu().numpy() - (p.Q * p.Q).T[:, cols])))
    print(f"{case}: max abs err vs Q o Q = {err:.3e}")
    return 0 if err <= 1e-10 else 1


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("gpu", "reference"), default="gpu")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle timing (profiling runs)")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the other workloads' records after the headline")
    ap.add_argument("--workload", choices=("planted1024", "batch4096", "planted4096", "goe64",
                                           "vectors1024", "herm1024", "single4002", "serving"),
                    default="planted1024",
                    help="planted1024 (default, the headline line); the others print a line "
                         "of the same shape for the other workloads")
    ap.add_argument("--serving-requests", type=int, default=40,
                    help="serving: length of the prefix of the seeded request stream")
    ap.add_argument("--serving-rates", default="0.5,1,2",
                    help="serving: comma-separated Poisson arrival rates (requests/s)")
    ap.add_argument("--profile-case", choices=("tridiag152", "tridiag304", "batch256", "single2002",
                                               "cluster2002", "herm512"), default=None,
                    help="run only a small case for an ncu capture and exit: tridiag152 / "
                         "tridiag304 = A plus the first 151 / 303 minors of the planted "
                         "n=1024 matrix (one / two CTAs per SM), called twice")
    args = ap.parse_args(argv)
    args.warmup = max(args.warmup, 3)   # timing rule: at least 3 untimed warm-up steps
    world, rank, local = dist_env()
    if args.profile_case:
        return run_profile_case(args.profile_case)
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.workload == "serving":
        return run_serving(args, world, rank, local)
    if args.workload != "planted1024":
        return run_other(args, world, rank, local)
    return run_gpu(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
